// rows_u8c1.cu -- the fused kernel's one-channel uint8 classes (3/8 K=8,
// 1/2 K=6, 2/3 K=6; Q14 taps, exact integer arithmetic), each in two tile
// shapes: shape 0 is the default measured on a B300, shape 1 the other
// pipeline depth (a candidate of the autotuner); shape 0 also for modular
// tilers.
#include "rows.cuh"

namespace ds {
namespace rows {
namespace {
//                      id           T        C  P  Q  K  NB  SR NST FP     PV QV KV FPW PRO   WPC MINB
using U8P_38_0 = Cls<kFcU8C1_38, uint8_t, 1, 3, 8, 8, 4,  8, 2, false, 3, 8, 8, 1, true,  1, 12>;
using U8P_38_1 = Cls<kFcU8C1_38, uint8_t, 1, 3, 8, 8, 4,  8, 3, false, 3, 8, 8, 1, true,  1, 8>;
using U8P_12_0 = Cls<kFcU8C1_12, uint8_t, 1, 1, 2, 6, 16, 4, 3, true,  1, 2, 6, 1, false, 1, 17>;
using U8P_12_1 = Cls<kFcU8C1_12, uint8_t, 1, 1, 2, 6, 16, 4, 2, true,  1, 2, 6, 1, false, 1, 17>;
using U8P_23_0 = Cls<kFcU8C1_23, uint8_t, 1, 2, 3, 6, 4,  3, 3, true,  2, 3, 6, 1, false, 4, 4>;
using U8P_23_1 = Cls<kFcU8C1_23, uint8_t, 1, 2, 3, 6, 4,  3, 2, true,  2, 3, 6, 1, false, 4, 4>;
}  // namespace

void register_u8c1(RowsTable& t) {
  t[kFcU8C1_38][0] = make_entry<U8P_38_0, true>();
  t[kFcU8C1_38][1] = make_entry<U8P_38_1, false>();
  t[kFcU8C1_12][0] = make_entry<U8P_12_0, true>();
  t[kFcU8C1_12][1] = make_entry<U8P_12_1, false>();
  t[kFcU8C1_23][0] = make_entry<U8P_23_0, true>();
  t[kFcU8C1_23][1] = make_entry<U8P_23_1, false>();
}

}  // namespace rows
}  // namespace ds
