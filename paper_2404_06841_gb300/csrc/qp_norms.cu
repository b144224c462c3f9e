// L^2_QP norms of differences of quasiperiodic functions given by their Fourier coefficients on K_N^n. By the
// Parseval identity of the L^2_QP norm (Sec. 2.2, eq. parseval) the norm is the l^2 norm of the coefficients,
// which is how Sec. 5.1 measures the error e_N = ||u_N - u||. Block partials in a fixed order, then one block
// sums them in a fixed order (deterministic, FP64).
#include "qp_device.cuh"

namespace qp {

// part[r * gridDim.x + block] = sum over the block's modes of |U_r - Uref_r|^2 (Uref may be null: |U_r|^2).
// hl > 0: half-spectrum storage with hl entries along the last axis; an entry off the plane k_{n-1} = 0 also
// stands for its mirror and counts twice.
__global__ void __launch_bounds__(BLOCK) k_sqdiff(int D, int nrhs, const double2* __restrict__ U,
                                                   const double2* __restrict__ Uref, double* part, int hl) {
  double v[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) v[r] = 0.0;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (r < nrhs) {
        double2 u = U[(size_t)r * D + e];
        if (Uref) {
          const double2 q = Uref[(size_t)r * D + e];
          u.x -= q.x;
          u.y -= q.y;
        }
        const double we = (hl > 0 && e % hl != 0) ? 2.0 : 1.0;
        v[r] = fma(we * u.x, u.x, fma(we * u.y, u.y, v[r]));
      }
    }
  }
  block_reduce<MAXR>(v);
  if (threadIdx.x == 0)
    for (int r = 0; r < nrhs; ++r) part[(size_t)r * gridDim.x + blockIdx.x] = v[r];
}

// out[r] = sqrt(sum of the nb partials of r), one block
__global__ void __launch_bounds__(BLOCK) k_sqdiff_final(int nb, int nrhs, const double* part, double* out) {
  double v[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) v[r] = 0.0;
  for (int i = threadIdx.x; i < nb; i += BLOCK)
#pragma unroll
    for (int r = 0; r < MAXR; ++r)
      if (r < nrhs) v[r] += part[(size_t)r * nb + i];
  block_reduce<MAXR>(v);
  if (threadIdx.x == 0)
    for (int r = 0; r < nrhs; ++r) out[r] = sqrt(v[r]);
}

// part: device, at least MAXR * nblk doubles; out: device, nrhs doubles; hl: as k_sqdiff (0: full spectrum).
void launch_l2_norms(int D, int nrhs, const double2* U, const double2* Uref, double* part, int nblk, double* out,
                     int hl, cudaStream_t s) {
  k_sqdiff<<<nblk, BLOCK, 0, s>>>(D, nrhs, U, Uref, part, hl);
  count_launch();
  k_sqdiff_final<<<1, BLOCK, 0, s>>>(nblk, nrhs, part, out);
  count_launch();
}

}  // namespace qp
