// rows_cif.cu -- the fused kernel's classes for the paper's CIF case (Sec. 3:
// 352 -> 132 per line, horizontal 3/8 K=8; 288 -> 128 lines, vertical 4/9
// K=8): uint8 RGB, and one uint8 plane (the planes of YUV 4:2:0).  Two
// frames per warp (16-lane strips), since a 352-pixel row is 44 packets.
// Each in two tile shapes: shape 0 is the default measured on a B300, shape
// 1 the other pipeline depth (RGB) or register budget (one plane), a
// candidate of the autotuner; shape 0 also for modular tilers.
#include "rows.cuh"

namespace ds {
namespace rows {
namespace {
//                      id            T        C  P  Q  K  NB SR NST FP     PV QV KV FPW PRO   WPC MINB
using U8_CIF_0  = Cls<kFcU8C3_CIF, uint8_t, 3, 3, 8, 8, 1, 9, 2, false, 4, 9, 8, 2, true, 1, 14>;
using U8_CIF_1  = Cls<kFcU8C3_CIF, uint8_t, 3, 3, 8, 8, 1, 9, 3, false, 4, 9, 8, 2, true, 1, 9>;
// the one-plane class: registers budgeted for 27 CTAs per SM (shared memory
// allows 31); shape 1 takes 31 (64 registers)
using U8P_CIF_0 = Cls<kFcU8C1_CIF, uint8_t, 1, 3, 8, 8, 1, 9, 2, true,  4, 9, 8, 2, true, 1, 27>;
using U8P_CIF_1 = Cls<kFcU8C1_CIF, uint8_t, 1, 3, 8, 8, 1, 9, 2, true,  4, 9, 8, 2, true, 1, 31>;
}  // namespace

void register_cif(RowsTable& t) {
  t[kFcU8C3_CIF][0] = make_entry<U8_CIF_0, true>();
  t[kFcU8C3_CIF][1] = make_entry<U8_CIF_1, false>();
  t[kFcU8C1_CIF][0] = make_entry<U8P_CIF_0, true>();
  t[kFcU8C1_CIF][1] = make_entry<U8P_CIF_1, false>();
}

}  // namespace rows
}  // namespace ds
