// Plain FP32 star-1 apply (qp_apply_stiffness) for the common fixed geometries, with the number of axes (every one
// carrying the taps m = +-e_j), d and the right-hand-side count compiled in: (n, d) = (6, 3), (4, 2), (2, 1) with
// d right-hand sides. The stencil's axis loop is then straight-line code and the compiler issues the neighbour
// reads of later axes early (cfg4's apply: 384 us against 435 with the geometry read at run time); the arithmetic
// and so the results are bit for bit those of the general star-1 kernel. The batch apply's variants are in
// qp_apply_fixed_batch.cu.
#include "qp_apply.cuh"

namespace qp {

namespace {

template <int NAX, int DC, bool REALC, int SK>
void plain_fixed(const StarParams& st, int nrhs, int D, const float2* h, float2* w, cudaStream_t s) {
  const int nblk = plain_star_grid<float, NAX>(D);
  if (st.hspec) k_apply_plain_star<float, REALC, DC, SK, NAX, DC, true><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w);
  else k_apply_plain_star<float, REALC, DC, SK, NAX, DC><<<nblk, BLOCK, 0, s>>>(st, D, nrhs, h, w);
}

template <int NAX, int DC>
void plain_fixed_any(bool realc, bool dg, const StarParams& st, int nrhs, int D, const float2* h, float2* w,
                     cudaStream_t s) {
  if (realc) {
    if (dg) plain_fixed<NAX, DC, true, 2>(st, nrhs, D, h, w, s);
    else plain_fixed<NAX, DC, true, 1>(st, nrhs, D, h, w, s);
  } else {
    if (dg) plain_fixed<NAX, DC, false, 2>(st, nrhs, D, h, w, s);
    else plain_fixed<NAX, DC, false, 1>(st, nrhs, D, h, w, s);
  }
}

}  // namespace

bool launch_plain_star_fixed(const StarParams& st, bool realc, int nrhs, int kind, int D, const float2* h, float2* w,
                             cudaStream_t s) {
  int n = 0;
  if (!fixed_geometry(st, nrhs, n)) return false;
  const bool dg = kind == QP_COEF_DIAG;
  if (n == 6) plain_fixed_any<6, 3>(realc, dg, st, nrhs, D, h, w, s);
  else if (n == 4) plain_fixed_any<4, 2>(realc, dg, st, nrhs, D, h, w, s);
  else plain_fixed_any<2, 1>(realc, dg, st, nrhs, D, h, w, s);
  return true;
}

}  // namespace qp
