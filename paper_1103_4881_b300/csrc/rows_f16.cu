// rows_f16.cu -- the fused kernel's fp16-storage classes (3/8 K=8, 1/2 K=6,
// 2/3 K=6; FP32 accumulation), each in two tile shapes: shape 0 is the
// default measured on a B300, shape 1 the other pipeline depth (2/3: the
// other register budget), a candidate of the autotuner; shape 0 also for
// modular tilers.
#include "rows.cuh"

namespace ds {
namespace rows {
namespace {
//                     id          T       C  P  Q  K  NB SR NST FP    PV QV KV FPW PRO   WPC MINB
using F16_38_0 = Cls<kFcF16_38, __half, 1, 3, 8, 8, 1, 8, 3, true, 3, 8, 8, 1, true,  1, 16>;
using F16_38_1 = Cls<kFcF16_38, __half, 1, 3, 8, 8, 1, 8, 2, true, 3, 8, 8, 1, true,  1, 16>;
using F16_12_0 = Cls<kFcF16_12, __half, 1, 1, 2, 6, 4, 8, 3, true, 1, 2, 6, 1, false, 1, 16>;
using F16_12_1 = Cls<kFcF16_12, __half, 1, 1, 2, 6, 4, 8, 2, true, 1, 2, 6, 1, false, 1, 16>;
// 2/3: registers budgeted for 26 CTAs per SM (shared memory allows 37), 2-5 %
// faster than 18 (shape 1) on 720p and 1080p batches
using F16_23_0 = Cls<kFcF16_23, __half, 1, 2, 3, 6, 2, 6, 2, true, 2, 3, 6, 1, false, 1, 26>;
using F16_23_1 = Cls<kFcF16_23, __half, 1, 2, 3, 6, 2, 6, 2, true, 2, 3, 6, 1, false, 1, 18>;
}  // namespace

void register_f16(RowsTable& t) {
  t[kFcF16_38][0] = make_entry<F16_38_0, true>();
  t[kFcF16_38][1] = make_entry<F16_38_1, false>();
  t[kFcF16_12][0] = make_entry<F16_12_0, true>();
  t[kFcF16_12][1] = make_entry<F16_12_1, false>();
  t[kFcF16_23][0] = make_entry<F16_23_0, true>();
  t[kFcF16_23][1] = make_entry<F16_23_1, false>();
}

}  // namespace rows
}  // namespace ds
