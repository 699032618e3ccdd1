// rows_f32.cu -- the fused kernel's fp32 classes (3/8 K=8, 1/2 K=6, 2/3 K=6),
// each in two tile shapes: shape 0 is the default measured on a B300, shape 1
// the other pipeline depth (a candidate of the autotuner); shape 0 also for
// modular tilers.
#include "rows.cuh"

namespace ds {
namespace rows {
namespace {
//                     id          T      C  P  Q  K  NB SR NST FP     PV QV KV FPW PRO    WPC MINB
using F32_38_0 = Cls<kFcF32_38, float, 1, 3, 8, 8, 1, 8, 2, false, 3, 8, 8, 1, false, 1, 12>;
using F32_38_1 = Cls<kFcF32_38, float, 1, 3, 8, 8, 1, 8, 3, false, 3, 8, 8, 1, false, 1, 8>;
using F32_12_0 = Cls<kFcF32_12, float, 1, 1, 2, 6, 4, 4, 3, true,  1, 2, 6, 1, false, 1, 17>;
using F32_12_1 = Cls<kFcF32_12, float, 1, 1, 2, 6, 4, 4, 2, true,  1, 2, 6, 1, false, 1, 17>;
using F32_23_0 = Cls<kFcF32_23, float, 1, 2, 3, 6, 2, 6, 3, true,  2, 3, 6, 1, false, 4, 4>;
using F32_23_1 = Cls<kFcF32_23, float, 1, 2, 3, 6, 2, 6, 2, true,  2, 3, 6, 1, false, 4, 4>;
}  // namespace

void register_f32(RowsTable& t) {
  t[kFcF32_38][0] = make_entry<F32_38_0, true>();
  t[kFcF32_38][1] = make_entry<F32_38_1, false>();
  t[kFcF32_12][0] = make_entry<F32_12_0, true>();
  t[kFcF32_12][1] = make_entry<F32_12_1, false>();
  t[kFcF32_23][0] = make_entry<F32_23_0, true>();
  t[kFcF32_23][1] = make_entry<F32_23_1, false>();
}

}  // namespace rows
}  // namespace ds
