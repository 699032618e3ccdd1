// rows_u8rgb.cu -- the fused kernel's uint8 RGB classes (3/8 K=8, 1/2 K=6,
// 2/3 K=6; Q14 taps, exact integer arithmetic), each in two tile shapes:
// shape 0 is the default measured on a B300, shape 1 the other pipeline
// depth (a candidate of the autotuner); shape 0 also for modular tilers.
#include "rows.cuh"

namespace ds {
namespace rows {
namespace {
//                     id           T        C  P  Q  K  NB SR NST FP    PV QV KV FPW PRO   WPC MINB
using U8_38_0 = Cls<kFcU8C3_38, uint8_t, 3, 3, 8, 8, 1, 8, 2, true, 3, 8, 8, 1, true,  1, 16>;
using U8_38_1 = Cls<kFcU8C3_38, uint8_t, 3, 3, 8, 8, 1, 8, 3, true, 3, 8, 8, 1, true,  1, 11>;
using U8_12_0 = Cls<kFcU8C3_12, uint8_t, 3, 1, 2, 6, 4, 4, 2, true, 1, 2, 6, 1, false, 1, 32>;
using U8_12_1 = Cls<kFcU8C3_12, uint8_t, 3, 1, 2, 6, 4, 4, 3, true, 1, 2, 6, 1, false, 1, 21>;
using U8_23_0 = Cls<kFcU8C3_23, uint8_t, 3, 2, 3, 6, 4, 3, 3, true, 2, 3, 6, 1, true,  1, 16>;
using U8_23_1 = Cls<kFcU8C3_23, uint8_t, 3, 2, 3, 6, 4, 3, 2, true, 2, 3, 6, 1, true,  1, 16>;
}  // namespace

void register_u8rgb(RowsTable& t) {
  t[kFcU8C3_38][0] = make_entry<U8_38_0, true>();
  t[kFcU8C3_38][1] = make_entry<U8_38_1, false>();
  t[kFcU8C3_12][0] = make_entry<U8_12_0, true>();
  t[kFcU8C3_12][1] = make_entry<U8_12_1, false>();
  t[kFcU8C3_23][0] = make_entry<U8_23_0, true>();
  t[kFcU8C3_23][1] = make_entry<U8_23_1, false>();
}

}  // namespace rows
}  // namespace ds
