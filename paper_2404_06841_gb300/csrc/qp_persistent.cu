// Host side of the persistent PCG solve (kernels in qp_persistent.cuh, instantiated per right-hand-side count
// in qp_persistent_nr*.cu): occupancy-bounded grid size and the cooperative launch.
#include "qp_internal.cuh"

namespace qp {

const void* persistent_kernel_nr1(bool realc);
const void* persistent_kernel_nr2(bool realc);
const void* persistent_kernel_nr3(bool realc);
const void* persistent_kernel_nr4(bool realc);
const void* persistent_star_kernel_nr1(bool realc, int sk);
const void* persistent_star_kernel_nr2(bool realc, int sk);
const void* persistent_star_kernel_nr3(bool realc, int sk);
const void* persistent_star_kernel_nr4(bool realc, int sk);
const void* persistent_star_fixed_kernel_n2(bool realc, int sk);
const void* persistent_star_fixed_kernel_n4(bool realc, int sk);
const void* persistent_star_fixed_kernel_n6(bool realc, int sk);

namespace {

// The instantiation for (realc, nr, sk); a star-1 plan of a fixed geometry (st) takes the one with its number of
// axes and d compiled in (bit for bit the same arithmetic).
const void* pick(bool realc, int nr, int sk, const StarParams* st) {
  int n = 0;
  if (sk != 0 && st && fixed_geometry(*st, nr, n)) {
    if (n == 6) return persistent_star_fixed_kernel_n6(realc, sk);
    if (n == 4) return persistent_star_fixed_kernel_n4(realc, sk);
    return persistent_star_fixed_kernel_n2(realc, sk);
  }
  if (sk != 0) {
    switch (nr) {
      case 1: return persistent_star_kernel_nr1(realc, sk);
      case 2: return persistent_star_kernel_nr2(realc, sk);
      case 3: return persistent_star_kernel_nr3(realc, sk);
      default: return persistent_star_kernel_nr4(realc, sk);
    }
  }
  switch (nr) {
    case 1: return persistent_kernel_nr1(realc);
    case 2: return persistent_kernel_nr2(realc);
    case 3: return persistent_kernel_nr3(realc);
    default: return persistent_kernel_nr4(realc);
  }
}

}  // namespace

size_t persistent_smem(int coef_count) { return (size_t)coef_count * (sizeof(double2) + sizeof(float2)); }

// Largest co-resident grid of the persistent solve for this instantiation (0: no cooperative launch).
int persistent_capacity(bool realc, int nr, int sk, const StarParams* st, size_t smem) {
  const void* fn = pick(realc, nr, sk, st);
  int dev = 0, coop = 0, sms = 0, per = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!coop) return 0;
  if (smem > 48 * 1024) CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, BLOCK, smem));
  return per * sms;
}

// Launches the persistent solve of one unit (b.single). bar (2 unsigned) and err (1 int) are device words
// zeroed here on the stream; grid must not exceed persistent_capacity (of the same realc, nr, sk, st).
void launch_persistent(const BatchDev& b, bool realc, int nr, int sk, const StarParams* st, int mode, bool warm,
                       unsigned* bar, int* err, double timeout_s, int grid, size_t smem, cudaStream_t s) {
  PersistArgs a;
  a.star = (sk != 0 && st) ? *st : StarParams{};
  a.b = b;
  a.bar = bar;
  a.err = err;
  a.mode = mode;
  a.warm = warm ? 1 : 0;
  a.timeout_ns = (unsigned long long)(timeout_s * 1e9);
  CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  void* args[] = {&a};
  CK(cudaLaunchCooperativeKernel(pick(realc, nr, sk, sk != 0 ? st : nullptr), dim3(grid), dim3(BLOCK), args, smem, s));
  count_launch();
}

}  // namespace qp
