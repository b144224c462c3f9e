// Batch FP32 (h, Q h) apply of the PCG iterations for a single star-1 unit of a fixed geometry, (n, d) = (6, 3),
// (4, 2), (2, 1) with taps on every axis and d right-hand sides: the number of axes and d compiled in, so the
// stencil's axis loop is straight-line code (as in qp_apply_fixed.cu). The arithmetic, the chunk walk and the
// reduction order are those of the general star-1 batch kernel, so the iterates are bit for bit the same.
#include "qp_apply.cuh"

namespace qp {

namespace {

// One resident block per slot (two per SM), each walking the chunks c, c + grid, ...: chunk c + k grid belongs to
// sweep wave k, so the resident blocks go through the waves in order; the per-chunk sums are those of any grid.
template <int NAX, int DC, bool REALC, int SK>
void batch_fixed(const BatchDev& b, int level, int refine, unsigned long long cond, int nblk, size_t smem,
                 const StarParams& st, cudaStream_t s) {
  nblk = std::min(nblk, sweep_chunks<float>());
  if (st.hspec)
    k_apply_star<float, EPI_DOT_HW, REALC, DC, SK, NAX, DC, true><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, st);
  else k_apply_star<float, EPI_DOT_HW, REALC, DC, SK, NAX, DC><<<nblk, BLOCK, smem, s>>>(b, level, refine, cond, st);
}

template <int NAX, int DC>
void batch_fixed_any(bool realc, bool dg, const BatchDev& b, int level, int refine, unsigned long long cond, int nblk,
                     size_t smem, const StarParams& st, cudaStream_t s) {
  if (realc) {
    if (dg) batch_fixed<NAX, DC, true, 2>(b, level, refine, cond, nblk, smem, st, s);
    else batch_fixed<NAX, DC, true, 1>(b, level, refine, cond, nblk, smem, st, s);
  } else {
    if (dg) batch_fixed<NAX, DC, false, 2>(b, level, refine, cond, nblk, smem, st, s);
    else batch_fixed<NAX, DC, false, 1>(b, level, refine, cond, nblk, smem, st, s);
  }
}

}  // namespace

bool launch_batch_star_fixed(const BatchDev& b, int level, int refine, unsigned long long cond, int nblk, size_t smem,
                             const StarParams& st, bool realc, int nr, int kind, cudaStream_t s) {
  int n = 0;
  if (!fixed_geometry(st, nr, n)) return false;
  const bool dg = kind == QP_COEF_DIAG;
  if (n == 6) batch_fixed_any<6, 3>(realc, dg, b, level, refine, cond, nblk, smem, st, s);
  else if (n == 4) batch_fixed_any<4, 2>(realc, dg, b, level, refine, cond, nblk, smem, st, s);
  else batch_fixed_any<2, 1>(realc, dg, b, level, refine, cond, nblk, smem, st, s);
  return true;
}

}  // namespace qp
