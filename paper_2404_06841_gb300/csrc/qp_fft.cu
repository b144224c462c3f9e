// n-dimensional complex DFT kernels and the FFT backend of the stiffness apply.
//
// Because the coefficient part A of Q = A o W is a multilevel circulant matrix (Sec. 4.1), the n-dim DFT
// diagonalises it and the apply of eq. n-discrete_equation becomes: gradient (multiply by lambda_b(k) = (P k)_b),
// unnormalised inverse DFT to the grid, pointwise product with A^{ab}(y_j) / D, forward DFT, divergence
// (multiply by lambda_a(k) and sum over a); the factors i and -i of gradient and divergence cancel.
//
// DFT: one pass per axis. A pass stages tiles of whole lines of that axis in shared memory (the rows of a tile
// are contiguous in memory, so loads and stores are coalesced), transforms each line in registers (radix 4/2/3
// decimation in time for N <= 32) or as N = N1 x N2 four-step through shared memory (N up to 1024), and writes
// the tile back. Twiddles for N <= 32 come from a constant-memory table filled once per device from host
// cos/sin; larger sizes call sincospi in the kernel.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qp_device.cuh"
#include "qp_fft.cuh"

namespace qp {

// ------------------------------------------------------------------------------------------------ twiddles

// Sizes transformed in registers and their offsets in the twiddle table (entries exp(2 pi i e / N), e < N).
constexpr int kSmall[] = {2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 27, 32};
constexpr int kNumSmall = sizeof(kSmall) / sizeof(int);
__host__ __device__ constexpr int tw_offset(int N) {
  int off = 0;
  for (int i = 0; i < kNumSmall; ++i) {
    if (kSmall[i] == N) return off;
    off += kSmall[i];
  }
  return -1;
}
constexpr int kTwTotal = tw_offset(32) + 32;

__constant__ double2 c_tw64[kTwTotal];
__constant__ float2 c_tw32[kTwTotal];

namespace {
std::mutex g_tw_mutex;
bool g_tw_ready[64] = {};
}  // namespace

// Fills the constant twiddle table on the current device (once per device).
static void ensure_twiddles() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_tw_mutex);
  if (dev >= 0 && dev < 64 && g_tw_ready[dev]) return;
  std::vector<double2> t64(kTwTotal);
  std::vector<float2> t32(kTwTotal);
  int off = 0;
  for (int i = 0; i < kNumSmall; ++i) {
    const int N = kSmall[i];
    for (int e = 0; e < N; ++e) {
      const long double ang = 2.0L * 3.14159265358979323846264338327950288L * (long double)e / (long double)N;
      const double c = (double)std::cos(ang), s = (double)std::sin(ang);
      t64[off + e] = make_double2(c, s);
      t32[off + e] = make_float2((float)c, (float)s);
    }
    off += N;
  }
  CK(cudaMemcpyToSymbol(c_tw64, t64.data(), kTwTotal * sizeof(double2)));
  CK(cudaMemcpyToSymbol(c_tw32, t32.data(), kTwTotal * sizeof(float2)));
  if (dev >= 0 && dev < 64) g_tw_ready[dev] = true;
}

template <typename T> __device__ __forceinline__ cplx<T> tw_at(int i);
template <> __device__ __forceinline__ double2 tw_at<double>(int i) { return c_tw64[i]; }
template <> __device__ __forceinline__ float2 tw_at<float>(int i) { return c_tw32[i]; }

template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// multiply by sign * i
template <typename T> __device__ __forceinline__ cplx<T> mul_si(cplx<T> a, int sign) {
  return sign > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
// W_N^{sign * e} from the table (e reduced mod N at compile time by the caller)
template <typename T, int N> __device__ __forceinline__ cplx<T> twd(int e, int sign) {
  constexpr int off = tw_offset(N);
  cplx<T> w = tw_at<T>(off + e % N);
  if (sign < 0) w.y = -w.y;
  return w;
}

// ------------------------------------------------------------------------------------------------ register DFT

// In-register DFT of N = 2^a 3^b <= 32 points: X_k = sum_n x_n exp(sign 2 pi i n k / N), by decimation in time
// with radix 4, 2 or 3 (all indices compile-time constants after unrolling).
template <typename T, int N>
struct RegDft {
  static __device__ __forceinline__ void run(cplx<T>* x, int sign) {
    constexpr int R = (N % 4 == 0 && N > 4) ? 4 : ((N % 2 == 0 && N > 2) ? 2 : ((N % 3 == 0 && N > 3) ? 3 : N));
    constexpr int M = N / R;
    cplx<T> sub[R][M];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int m = 0; m < M; ++m) sub[r][m] = x[r + R * m];
#pragma unroll
    for (int r = 0; r < R; ++r) RegDft<T, M>::run(sub[r], sign);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      cplx<T> t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = (r * k == 0) ? sub[r][k] : cmul<T>(sub[r][k], twd<T, N>(r * k, sign));
      RegDft<T, R>::run(t, sign);
#pragma unroll
      for (int q = 0; q < R; ++q) x[k + M * q] = t[q];
    }
  }
};
template <typename T> struct RegDft<T, 1> {
  static __device__ __forceinline__ void run(cplx<T>*, int) {}
};
template <typename T> struct RegDft<T, 2> {
  static __device__ __forceinline__ void run(cplx<T>* x, int) {
    const cplx<T> a = x[0], b = x[1];
    x[0] = cadd<T>(a, b);
    x[1] = csub<T>(a, b);
  }
};
template <typename T> struct RegDft<T, 3> {
  static __device__ __forceinline__ void run(cplx<T>* x, int sign) {
    // X_k = x0 + x1 w^k + x2 w^{2k}, w = exp(sign 2 pi i / 3) = -1/2 + sign i sqrt(3)/2
    const cplx<T> w1 = twd<T, 3>(1, sign);
    const cplx<T> s = cadd<T>(x[1], x[2]), d = csub<T>(x[1], x[2]);
    const cplx<T> a = x[0];
    x[0] = cadd<T>(a, s);
    const cplx<T> m = mk<T>(a.x + w1.x * s.x, a.y + w1.x * s.y);       // a - s/2
    const cplx<T> j = mk<T>(-w1.y * d.y, w1.y * d.x);                 // i * (sign sqrt3/2) * d
    x[1] = cadd<T>(m, j);
    x[2] = csub<T>(m, j);
  }
};
template <typename T> struct RegDft<T, 4> {
  static __device__ __forceinline__ void run(cplx<T>* x, int sign) {
    const cplx<T> a = cadd<T>(x[0], x[2]), b = csub<T>(x[0], x[2]);
    const cplx<T> c = cadd<T>(x[1], x[3]), e = mul_si<T>(csub<T>(x[1], x[3]), sign);
    x[0] = cadd<T>(a, c);
    x[2] = csub<T>(a, c);
    x[1] = cadd<T>(b, e);
    x[3] = csub<T>(b, e);
  }
};

// ------------------------------------------------------------------------------------------------ axis pass

// One DFT pass along one axis of `count` arrays seen as [outer O][N][inner I] (C order). A block handles
// L x R lines: L consecutive outer indices times R consecutive inner indices; the tile [L][N][R] is staged in
// shared memory. Each thread transforms whole lines (in registers for N <= 32).
template <typename T, int N>
__global__ void __launch_bounds__(BLOCK) k_fft_axis(cplx<T>* data, long long O, int I, int L, int R, int sign) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smraw);
  const long long nI = (I + R - 1) / R;          // inner blocks per outer row
  const long long nO = (O + L - 1) / L;
  const long long blk = blockIdx.x + (long long)blockIdx.y * gridDim.x;
  if (blk >= nO * nI) return;
  const long long o0 = (blk / nI) * L;
  const int i0 = (int)(blk % nI) * R;
  const int lrows = (int)min((long long)L, O - o0), rcols = min(R, I - i0);
  const int tsz = L * N * R;
  // load: element (l, k, r) at ((o0 + l) * N + k) * I + i0 + r; rows of r are contiguous
  for (int t = threadIdx.x; t < tsz; t += BLOCK) {
    const int r = t % R, k = (t / R) % N, l = t / (R * N);
    if (l < lrows && r < rcols) tile[t] = data[((o0 + l) * N + k) * (long long)I + i0 + r];
  }
  __syncthreads();
  for (int line = threadIdx.x; line < L * R; line += BLOCK) {
    const int l = line / R, r = line % R;
    if (l < lrows && r < rcols) {
      cplx<T> x[N];
#pragma unroll
      for (int k = 0; k < N; ++k) x[k] = tile[(l * N + k) * R + r];
      RegDft<T, N>::run(x, sign);
#pragma unroll
      for (int k = 0; k < N; ++k) tile[(l * N + k) * R + r] = x[k];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < tsz; t += BLOCK) {
    const int r = t % R, k = (t / R) % N, l = t / (R * N);
    if (l < lrows && r < rcols) data[((o0 + l) * N + k) * (long long)I + i0 + r] = tile[t];
  }
}

// Same pass for N = N1 * N2 (both <= 32): with n = n1 + N1 n2 and k = k2 + N2 k1,
// X[k] = sum_{n1} W_N^{n1 k2} W_{N1}^{n1 k1} sum_{n2} x[n1 + N1 n2] W_{N2}^{n2 k2}.
// Step A transforms along n2 (stride N1), step B applies W_N^{n1 k2} (sincospi), step C transforms along n1 and
// leaves X[k2 + N2 k1] at tile position k1 + N1 k2; the store maps positions back to natural order.
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(BLOCK) k_fft_axis_2(cplx<T>* data, long long O, int I, int L, int R, int sign) {
  constexpr int N = N1 * N2;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smraw);
  const long long nI = (I + R - 1) / R;
  const long long nO = (O + L - 1) / L;
  const long long blk = blockIdx.x + (long long)blockIdx.y * gridDim.x;
  if (blk >= nO * nI) return;
  const long long o0 = (blk / nI) * L;
  const int i0 = (int)(blk % nI) * R;
  const int lrows = (int)min((long long)L, O - o0), rcols = min(R, I - i0);
  const int tsz = L * N * R;
  for (int t = threadIdx.x; t < tsz; t += BLOCK) {
    const int r = t % R, k = (t / R) % N, l = t / (R * N);
    if (l < lrows && r < rcols) tile[t] = data[((o0 + l) * N + k) * (long long)I + i0 + r];
  }
  __syncthreads();
  // step A + B: per (n1, line), line fastest so that neighbouring threads touch neighbouring r
  const int LR = L * R;
  for (int job = threadIdx.x; job < LR * N1; job += BLOCK) {
    const int line = job % LR, n1 = job / LR, l = line / R, r = line % R;
    if (l < lrows && r < rcols) {
      cplx<T> x[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) x[n2] = tile[(l * N + n1 + N1 * n2) * R + r];
      RegDft<T, N2>::run(x, sign);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        cplx<T> v = x[k2];
        if (n1 * k2 != 0) {
          T sv, cv;
          if (sizeof(T) == 8) {
            double s_, c_;
            sincospi(2.0 * (double)((n1 * k2) % N) / (double)N, &s_, &c_);
            sv = (T)s_;
            cv = (T)c_;
          } else {
            float s_, c_;
            sincospif(2.0f * (float)((n1 * k2) % N) / (float)N, &s_, &c_);
            sv = (T)s_;
            cv = (T)c_;
          }
          v = cmul<T>(v, mk<T>(cv, sign > 0 ? sv : -sv));
        }
        tile[(l * N + n1 + N1 * k2) * R + r] = v;
      }
    }
  }
  __syncthreads();
  // step C: per (k2, line); X[k2 + N2 k1] goes straight to global memory (rows of r stay contiguous)
  for (int job = threadIdx.x; job < LR * N2; job += BLOCK) {
    const int line = job % LR, k2 = job / LR, l = line / R, r = line % R;
    if (l < lrows && r < rcols) {
      cplx<T> x[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) x[n1] = tile[(l * N + n1 + N1 * k2) * R + r];
      RegDft<T, N1>::run(x, sign);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) data[((o0 + l) * N + k2 + N2 * k1) * (long long)I + i0 + r] = x[k1];
    }
  }
}

// Tile shape: about 8 KB (FP32) / 16 KB (FP64) of lines per block, rows of R >= 4 contiguous elements.
static void tile_shape(int N, long long O, int I, int& L, int& R) {
  const int target = 2048;                 // elements per tile
  if (I >= 8) {
    R = std::min(I, std::max(8, target / N));
    R = std::min(R, 64);
    L = 1;
  } else {
    R = I;
    L = (int)std::max<long long>(1, std::min<long long>(O, std::max(1, target / (N * I))));
  }
}

template <typename T, int N>
static void axis_small(cplx<T>* data, long long O, int I, int sign, cudaStream_t s) {
  int L, R;
  tile_shape(N, O, I, L, R);
  const long long blocks = ((O + L - 1) / L) * ((I + R - 1) / R);
  const size_t smem = (size_t)L * N * R * sizeof(cplx<T>);
  dim3 grid((unsigned)std::min<long long>(blocks, 65535), (unsigned)((blocks + 65534) / 65535));
  k_fft_axis<T, N><<<grid, BLOCK, smem, s>>>(data, O, I, L, R, sign);
  count_launch();
}

template <typename T, int N1, int N2>
static void axis_two(cplx<T>* data, long long O, int I, int sign, cudaStream_t s) {
  constexpr int N = N1 * N2;
  int L = 1, R = 1;
  const int target = (sizeof(T) == 8 ? 2048 : 4096);
  if (I >= 4) {
    R = std::min(I, std::max(4, target / N));
    L = 1;
  } else {
    R = I;
    L = (int)std::max<long long>(1, std::min<long long>(O, std::max(1, target / (N * I))));
  }
  const long long blocks = ((O + L - 1) / L) * ((I + R - 1) / R);
  const size_t smem = (size_t)L * N * R * sizeof(cplx<T>);
  if (smem > 200 * 1024) raise(QP_ERR_UNSUPPORTED, "FFT tile exceeds shared memory");
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_fft_axis_2<T, N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)std::min<long long>(blocks, 65535), (unsigned)((blocks + 65534) / 65535));
  k_fft_axis_2<T, N1, N2><<<grid, BLOCK, smem, s>>>(data, O, I, L, R, sign);
  count_launch();
}

// True if the library's FFT kernels transform an axis of size N.
bool fft_supported(int N) {
  switch (N) {
    case 2: case 3: case 4: case 6: case 8: case 9: case 12: case 16: case 18: case 24: case 27: case 32:
    case 48: case 64: case 72: case 96: case 128: case 144: case 192: case 256: case 288: case 384: case 512:
    case 576: case 768: case 1024:
      return true;
    default:
      return false;
  }
}

// One pass along an axis of size N with inner size I (product of the later axes) and outer size O.
template <typename T>
static void fft_axis(cplx<T>* data, int N, long long O, int I, int sign, cudaStream_t s) {
  switch (N) {
    case 2: axis_small<T, 2>(data, O, I, sign, s); break;
    case 3: axis_small<T, 3>(data, O, I, sign, s); break;
    case 4: axis_small<T, 4>(data, O, I, sign, s); break;
    case 6: axis_small<T, 6>(data, O, I, sign, s); break;
    case 8: axis_small<T, 8>(data, O, I, sign, s); break;
    case 9: axis_small<T, 9>(data, O, I, sign, s); break;
    case 12: axis_small<T, 12>(data, O, I, sign, s); break;
    case 16: axis_small<T, 16>(data, O, I, sign, s); break;
    case 18: axis_small<T, 18>(data, O, I, sign, s); break;
    case 24: axis_small<T, 24>(data, O, I, sign, s); break;
    case 27: axis_small<T, 27>(data, O, I, sign, s); break;
    case 32: axis_small<T, 32>(data, O, I, sign, s); break;
    case 48: axis_two<T, 16, 3>(data, O, I, sign, s); break;
    case 64: axis_two<T, 8, 8>(data, O, I, sign, s); break;
    case 72: axis_two<T, 8, 9>(data, O, I, sign, s); break;
    case 96: axis_two<T, 32, 3>(data, O, I, sign, s); break;
    case 128: axis_two<T, 16, 8>(data, O, I, sign, s); break;
    case 144: axis_two<T, 16, 9>(data, O, I, sign, s); break;
    case 192: axis_two<T, 32, 6>(data, O, I, sign, s); break;
    case 256: axis_two<T, 16, 16>(data, O, I, sign, s); break;
    case 288: axis_two<T, 32, 9>(data, O, I, sign, s); break;
    case 384: axis_two<T, 32, 12>(data, O, I, sign, s); break;
    case 512: axis_two<T, 32, 16>(data, O, I, sign, s); break;
    case 576: axis_two<T, 32, 18>(data, O, I, sign, s); break;
    case 768: axis_two<T, 32, 24>(data, O, I, sign, s); break;
    case 1024: axis_two<T, 32, 32>(data, O, I, sign, s); break;
    default: raise(QP_ERR_UNSUPPORTED, "FFT size " + std::to_string(N) + " is not built");
  }
}

// In-place unnormalised n-dim DFT of `count` contiguous arrays of shape N[0..n-1].
template <typename T>
static void fft_nd(cplx<T>* data, int n, const int* N, long long count, int sign, cudaStream_t s) {
  ensure_twiddles();
  long long D = 1;
  for (int j = 0; j < n; ++j) D *= N[j];
  for (int j = 0; j < n; ++j) {
    long long inner = 1;
    for (int t = j + 1; t < n; ++t) inner *= N[t];
    const long long outer = count * D / (inner * N[j]);
    if (inner > (1ll << 30)) raise(QP_ERR_UNSUPPORTED, "inner size too large");
    fft_axis<T>(data, N[j], outer, (int)inner, sign, s);
  }
}

void fft_standalone(int n, const int* N, int count, void* data, int sign, int precision, cudaStream_t s) {
  for (int j = 0; j < n; ++j)
    if (!fft_supported(N[j])) raise(QP_ERR_UNSUPPORTED, "FFT size " + std::to_string(N[j]) + " is not built");
  if (precision == QP_FP64) fft_nd<double>(static_cast<double2*>(data), n, N, count, sign, s);
  else fft_nd<float>(static_cast<float2*>(data), n, N, count, sign, s);
}

// ------------------------------------------------------------------------------------------------ FFT backend

// A pass of the fused apply over one group of consecutive axes (kernels below).
struct GroupPass {
  int mode;                 // GP_*
  int sign;                 // GP_PLAIN: +1 inverse, -1 forward
  int ng, j0;               // axes j0 .. j0 + ng - 1
  int Ng[MAXN], sg[MAXN];   // their sizes; stride of each in the group position (product of later group axes)
  int nhi[MAXN];            // M / (Ng * sg): group positions above each axis
  FastDiv fR;               // tile element -> (l M + pos, r)
  FastDiv fsg[MAXN], fnhi[MAXN];
  int M, I, L, R, TS, ntile;
  long long O;
  int tiles_o, tiles_i;
  // aff: the array index of tile element idx + BLOCK is that of idx plus dlin for every idx of the tile, so a
  // thread's elements idx = t, t + BLOCK, ... sit at lin(t) + u dlin (no per-element division)
  int aff, dlin;
  size_t smem;
};

enum { GP_GRAD_INV = 0, GP_PLAIN = 1, GP_INV_COEF_FWD = 2, GP_FWD_DIV = 3, GP_SINGLE = 4 };

struct FusedSchedule {
  bool ok = false;            // false: the per-axis path (gradient, n-dim FFT, coefficient, FFT, divergence)
  int npass = 0;
  int kb = 0;                 // tile budget (KB of shared memory per block) the passes were sized for
  GroupPass pass[5];
};

// The FFT-backend apply's candidate schedules for one precision, the one in use, and the autotuner's timings.
struct ScheduleSet {
  std::vector<FusedSchedule> cand;   // deterministic order; the last one is the per-axis path
  std::vector<float> ms;             // measured ms per apply (empty: not tuned)
  int chosen = -1;
};

struct FftPlan {
  int d = 0, n = 0, D = 0, ncomp = 0, kind = 0, max_rhs = 0, precisions = 3;
  int N[MAXN] = {};
  std::vector<void*> allocs;
  int64_t bytes = 0;
  double* coef64 = nullptr;     // A^{c}(y_j) / D, [ncomp][D]
  float* coef32 = nullptr;
  double2* ahat = nullptr;      // A~^{c}_k, [ncomp][D] (FP64)
  double2* f64 = nullptr;       // fields [d][max_rhs][D]
  float2* f32 = nullptr;
  double* part = nullptr;       // reduction partials
  int nblk = 0;
  FusedSchedule fused64, fused32;   // group-pass schedules of the apply (ok = false: per-axis passes)
  ScheduleSet sched64, sched32;     // their candidates (autotuner)
  cudaStream_t stream = nullptr;   // the creating stream (allocations are ordered on it)
  void* take(size_t b) {
    void* p = dev_alloc(b, stream);
    allocs.push_back(p);
    bytes += (int64_t)b;
    return p;
  }
  ~FftPlan() {
    for (void* p : allocs) dev_free(p);
  }
};

static FusedSchedule plan_fused(const PlanDev& pd, int esize, int kb = 100);
static std::vector<FusedSchedule> fused_candidates(const PlanDev& pd, int esize);

FftPlan* fft_plan_create(const PlanDev& pd, int precisions, int max_rhs, cudaStream_t s) {
  for (int j = 0; j < pd.n; ++j)
    if (!fft_supported(pd.N[j])) raise(QP_ERR_UNSUPPORTED, "FFT size " + std::to_string(pd.N[j]) + " is not built");
  ensure_twiddles();
  FftPlan* f = new FftPlan();
  f->stream = s;
  try {
    f->d = pd.d;
    f->n = pd.n;
    f->D = pd.D;
    f->ncomp = pd.ncomp;
    f->kind = pd.kind;
    f->max_rhs = max_rhs;
    f->precisions = precisions;
    for (int j = 0; j < pd.n; ++j) f->N[j] = pd.N[j];
    const size_t D = (size_t)pd.D;
    f->coef64 = (double*)f->take(D * pd.ncomp * sizeof(double));
    f->coef32 = (float*)f->take(D * pd.ncomp * sizeof(float));
    f->ahat = (double2*)f->take(D * pd.ncomp * sizeof(double2));
    if (precisions & 1) f->f64 = (double2*)f->take(D * pd.d * max_rhs * sizeof(double2));
    else f->f64 = (double2*)f->take(D * sizeof(double2));   // set-up transforms only
    if (precisions & 2) f->f32 = (float2*)f->take(D * pd.d * max_rhs * sizeof(float2));
    f->nblk = (int)std::min<int64_t>((pd.D + BLOCK - 1) / BLOCK, 152 * 8);
    f->fused64 = plan_fused(pd, (int)sizeof(double2));
    f->fused32 = plan_fused(pd, (int)sizeof(float2));
    f->sched64.cand = fused_candidates(pd, (int)sizeof(double2));
    f->sched32.cand = fused_candidates(pd, (int)sizeof(float2));
    f->part = (double*)f->take((size_t)f->nblk * 2 * MAXD * MAXD * sizeof(double) + 1024);
  } catch (...) {
    delete f;
    throw;
  }
  return f;
}

void fft_plan_destroy(FftPlan* f) { delete f; }
int64_t fft_plan_bytes(const FftPlan* f) { return f ? f->bytes : 0; }

// lambda_a(k) for the mode at linear index e.
template <typename T>
__device__ __forceinline__ void lambda_of(const PlanDev& p, int e, T (&lk)[MAXD], int (&ib)[MAXN]) {
  int k[MAXN];
  mode_digits(p, e, ib, k);
#pragma unroll
  for (int a = 0; a < MAXD; ++a) {
    lk[a] = T(0);
#pragma unroll
    for (int j = 0; j < MAXN; ++j)
      if (a < p.d && j < p.n) lk[a] = fma(pcoef<T>(p, a, j), (T)k[j], lk[a]);
  }
}

// coefficient entry (a, b) from the stored components at node e
template <typename T>
__device__ __forceinline__ T coef_at(int kind, int d, const T* c, int D, int e, int a, int b) {
  if (kind == QP_COEF_SCALAR) return a == b ? c[e] : T(0);
  if (kind == QP_COEF_DIAG) return a == b ? c[(size_t)a * D + e] : T(0);
  return c[(size_t)sym_idx(a, b, d) * D + e];
}

// entry (a, b) of A from the components c[0 .. ncomp) of one node (scalar / diagonal / upper triangle)
constexpr int MAXC = MAXD * (MAXD + 1) / 2;
// The d x d matrix from the components of one node, with compile-time indices only (registers, no stack).
template <typename T>
__device__ __forceinline__ void fill_matrix(int kind, int d, const T (&c)[MAXC], T (&A)[MAXD][MAXD]) {
#pragma unroll
  for (int a = 0; a < MAXD; ++a)
#pragma unroll
    for (int b = 0; b < MAXD; ++b) A[a][b] = T(0);
  if (kind == QP_COEF_SCALAR) {
    A[0][0] = A[1][1] = A[2][2] = c[0];
  } else if (kind == QP_COEF_DIAG) {
    A[0][0] = c[0];
    A[1][1] = c[1];
    A[2][2] = c[2];
  } else if (d == 1) {
    A[0][0] = c[0];
  } else if (d == 2) {
    A[0][0] = c[0];
    A[0][1] = A[1][0] = c[1];
    A[1][1] = c[2];
  } else {
    A[0][0] = c[0];
    A[0][1] = A[1][0] = c[1];
    A[0][2] = A[2][0] = c[2];
    A[1][1] = c[3];
    A[1][2] = A[2][1] = c[4];
    A[2][2] = c[5];
  }
}

// set-up: real grid samples -> complex buffer (component c), and the scaled FP64 / FP32 copies A / D
__global__ void k_grid_prepare(const PlanDev* pdp, const double* grid, int comp, double2* z, double* c64, float* c32) {
  const PlanDev& p = *pdp;
  const int D = p.D;
  const double inv = 1.0 / (double)D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    const double v = grid[(size_t)comp * D + e];
    z[e] = make_double2(v, 0.0);
    c64[(size_t)comp * D + e] = v * inv;
    c32[(size_t)comp * D + e] = (float)(v * inv);
  }
}

__global__ void k_scale_store(const double2* z, double2* out, int D, double s) {
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    const double2 v = z[e];
    out[e] = make_double2(v.x * s, v.y * s);
  }
}

void fft_set_grid(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const double* grid, cudaStream_t s) {
  for (int c = 0; c < f->ncomp; ++c) {
    k_grid_prepare<<<f->nblk, BLOCK, 0, s>>>(pdp, grid, c, f->f64, f->coef64, f->coef32);
    count_launch();
    fft_nd<double>(f->f64, pd.n, pd.N, 1, -1, s);
    k_scale_store<<<f->nblk, BLOCK, 0, s>>>(f->f64, f->ahat + (size_t)c * pd.D, pd.D, 1.0 / (double)pd.D);
    count_launch();
  }
  CK_LAUNCH();
}

// set-up from taps: scatter A~ to the table, inverse DFT (unnormalised) gives the grid samples
__global__ void k_scatter_taps(const PlanDev* pdp, int comp, double2* ahat) {
  const PlanDev& p = *pdp;
  for (int t = threadIdx.x; t < p.ntaps; t += blockDim.x) {
    int e = 0;
    for (int ax = 0; ax < p.n; ++ax) {
      const int mj = p.m[t][ax];
      e += (mj < 0 ? mj + p.N[ax] : mj) * p.stride[ax];
    }
    ahat[(size_t)comp * p.D + e] = p.coef64[(size_t)t * p.ncomp + comp];
  }
}

__global__ void k_grid_from_z(const PlanDev* pdp, const double2* z, int comp, double* c64, float* c32) {
  const PlanDev& p = *pdp;
  const int D = p.D;
  const double inv = 1.0 / (double)D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    const double v = z[e].x;
    c64[(size_t)comp * D + e] = v * inv;
    c32[(size_t)comp * D + e] = (float)(v * inv);
  }
}

void fft_set_taps(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, cudaStream_t s) {
  CK(cudaMemsetAsync(f->ahat, 0, (size_t)f->ncomp * pd.D * sizeof(double2), s));
  for (int c = 0; c < f->ncomp; ++c) {
    k_scatter_taps<<<1, BLOCK, 0, s>>>(pdp, c, f->ahat);
    count_launch();
    CK(cudaMemcpyAsync(f->f64, f->ahat + (size_t)c * pd.D, (size_t)pd.D * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    fft_nd<double>(f->f64, pd.n, pd.N, 1, +1, s);
    k_grid_from_z<<<f->nblk, BLOCK, 0, s>>>(pdp, f->f64, c, f->coef64, f->coef32);
    count_launch();
  }
  CK_LAUNCH();
}

// Jacobi diagonal q(k) = lambda(k)^T A~_0 lambda(k); the Frobenius diagonal is built on first use
// (fft_frobenius; frob = 0 until then). Reduces min |lambda|^2 and min q/|lambda|^2 over k != 0 and the smallest Cholesky pivot of
// A over the grid nodes into partials; k_diag_fft_final writes out[0..2].
__global__ void __launch_bounds__(BLOCK) k_diag_fft(const PlanDev* pdp, const double2* ahat, const double* c64,
                                                    double* jac, double* frob, float* jac32, float* frob32,
                                                    double* part) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d;
  double a0[MAXD][MAXD];
  for (int a = 0; a < MAXD; ++a)
    for (int b = 0; b < MAXD; ++b) {
      double v = 0.0;
      if (a < d && b < d) {
        if (p.kind == QP_COEF_SCALAR) v = (a == b) ? ahat[0].x : 0.0;
        else if (p.kind == QP_COEF_DIAG) v = (a == b) ? ahat[(size_t)a * D].x : 0.0;
        else v = ahat[(size_t)sym_idx(a, b, d) * D].x;
      }
      a0[a][b] = v;
    }
  double red[3] = {DBL_MAX, DBL_MAX, DBL_MAX};
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    double q = 0.0, l2 = 0.0;
    for (int a = 0; a < d; ++a) {
      l2 += lk[a] * lk[a];
      for (int b = 0; b < d; ++b) q += lk[a] * a0[a][b] * lk[b];
    }
    double mj = 0.0;
    if (e != 0) {
      mj = q != 0.0 ? 1.0 / q : 0.0;
      red[0] = fmin(red[0], l2);
      red[1] = fmin(red[1], l2 > 0.0 ? q / l2 : -1.0);
    }
    jac[e] = mj;
    frob[e] = 0.0;
    jac32[e] = (float)mj;
    frob32[e] = 0.0f;
    // Cholesky pivots of A(y_e) = D * coef (symmetric d x d)
    double A[MAXD][MAXD], L[MAXD][MAXD];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) A[a][b] = coef_at<double>(p.kind, d, c64, D, e, a, b) * (double)D;
    double piv = DBL_MAX;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j <= i; ++j) {
        double sdot = A[i][j];
        for (int k = 0; k < j; ++k) sdot -= L[i][k] * L[j][k];
        if (i == j) {
          piv = fmin(piv, sdot);
          L[i][i] = sdot > 0.0 ? sqrt(sdot) : 1.0;
        } else {
          L[i][j] = sdot / L[j][j];
        }
      }
    red[2] = fmin(red[2], piv);
  }
  block_reduce<3, true>(red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = red[q];
}

__global__ void k_diag_fft_final(const double* part, int nb, double* out) {
  double v[3] = {DBL_MAX, DBL_MAX, DBL_MAX};
  for (int i = threadIdx.x; i < nb; i += BLOCK)
    for (int q = 0; q < 3; ++q) v[q] = fmin(v[q], part[(size_t)q * nb + i]);
  block_reduce<3, true>(v);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) out[q] = v[q];
}

void fft_diag(FftPlan* f, const PlanDev*, const PlanDev* pdp, double* jac, double* frob, float* jac32, float* frob32,
              double* out, cudaStream_t s) {
  k_diag_fft<<<f->nblk, BLOCK, 0, s>>>(pdp, f->ahat, f->coef64, jac, frob, jac32, frob32, f->part);
  k_diag_fft_final<<<1, BLOCK, 0, s>>>(f->part, f->nblk, out);
  count_launch(2);
  CK_LAUNCH();
}

// ---- Frobenius-optimal diagonal (Sec. 4.3, eq. preconditioner) on the FFT backend
//
// M(k) = q(k) / ||Q e_k||^2 with q(k) = lambda(k)^T A~_0 lambda(k). Column k of Q holds, at row k + m (mod N),
// e_m(k) = sum_ab lambda_a(k + m) A~^{ab}_m lambda_b(k), so
//   ||Q e_k||^2 = sum_{b,b'} lambda_b(k) lambda_b'(k) sum_{a,a'} sum_m G^{aa'}(k + m) H^{ab,a'b'}(m),
//   G^{aa'} = lambda_a lambda_a',  H^{ab,a'b'}(m) = A~^{ab}_m conj(A~^{a'b'}_m),
// and each inner sum over all D modes m is a circular cross-correlation on the mode grid: with
// Hr(z) = H(-z), sum_m G(k + m) H(m) = (G * Hr)(k) = DFT^-1(DFT(G) DFT(Hr))(k) / D. With a dense coefficient
// this costs d^4 + d(d+1) FP64 n-dim DFTs instead of the O(D^2) direct sum.

__device__ __forceinline__ int coef_comp(int kind, int d, int a, int b) {
  if (kind == QP_COEF_SCALAR) return a == b ? 0 : -1;
  if (kind == QP_COEF_DIAG) return a == b ? a : -1;
  return sym_idx(a, b, d);
}

// G(e) = lambda_a(e) lambda_a'(e)
__global__ void __launch_bounds__(BLOCK) k_fro_g(const PlanDev* pdp, int a, int a2, double2* G) {
  const PlanDev& p = *pdp;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < p.D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    G[e] = make_double2(lk[a] * lk[a2], 0.0);
  }
}

// Hr(e) = A~^{c1}(-e) conj(A~^{c2}(-e)), -e the mode with every storage digit negated mod N_j
__global__ void __launch_bounds__(BLOCK) k_fro_h(const PlanDev* pdp, const double2* ahat, int c1, int c2,
                                                 double2* H) {
  const PlanDev& p = *pdp;
  const int D = p.D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    int ib[MAXN], k[MAXN];
    mode_digits(p, e, ib, k);
    int en = 0;
    for (int j = 0; j < p.n; ++j) en += (ib[j] == 0 ? 0 : p.N[j] - ib[j]) * p.stride[j];
    const double2 x = ahat[(size_t)c1 * D + en], y = ahat[(size_t)c2 * D + en];
    H[e] = make_double2(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y);
  }
}

// X += A B (complex, elementwise)
__global__ void __launch_bounds__(BLOCK) k_fro_macc(int D, const double2* A, const double2* B, double2* X) {
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    const double2 a = A[e], b = B[e];
    double2 x = X[e];
    x.x = fma(a.x, b.x, fma(-a.y, b.y, x.x));
    x.y = fma(a.x, b.y, fma(a.y, b.x, x.y));
    X[e] = x;
  }
}

// cn(e) += lambda_b(e) lambda_b'(e) Re(X(e)) / D
__global__ void __launch_bounds__(BLOCK) k_fro_cn(const PlanDev* pdp, int b, int b2, const double2* X, double* cn) {
  const PlanDev& p = *pdp;
  const double invD = 1.0 / (double)p.D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < p.D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    cn[e] = fma(lk[b] * lk[b2], X[e].x * invD, cn[e]);
  }
}

// M(k) = q(k) / ||Q e_k||^2 (0 at k = 0 and where the column vanishes), FP64 and FP32 copies
__global__ void __launch_bounds__(BLOCK) k_fro_final(const PlanDev* pdp, const double2* ahat, const double* cn,
                                                     double* frob, float* frob32) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    double q = 0.0;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        const int c = coef_comp(p.kind, d, a, b);
        if (c >= 0) q += lk[a] * ahat[(size_t)c * D].x * lk[b];
      }
    const double m = (e != 0 && cn[e] > 0.0) ? q / cn[e] : 0.0;
    frob[e] = m;
    frob32[e] = (float)m;
  }
}

void fft_frobenius(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, double* frob, float* frob32, cudaStream_t s) {
  const int d = pd.d, kind = pd.kind;
  const size_t D = (size_t)pd.D;
  const int npair = d * (d + 1) / 2;
  std::vector<void*> tmp;
  auto take = [&](size_t bytes) {
    void* q = dev_alloc(bytes, s);
    tmp.push_back(q);
    return q;
  };
  try {
    double2* G = (double2*)take(npair * D * sizeof(double2));
    double2* H = (double2*)take(D * sizeof(double2));
    double2* X = (double2*)take(D * sizeof(double2));
    double* cn = (double*)take(D * sizeof(double));
    CK(cudaMemsetAsync(cn, 0, D * sizeof(double), s));
    auto pidx = [&](int a, int a2) {   // index of the unordered pair (min, max)
      const int lo = std::min(a, a2), hi = std::max(a, a2);
      return lo * d - lo * (lo - 1) / 2 + (hi - lo);
    };
    for (int a = 0; a < d; ++a)
      for (int a2 = a; a2 < d; ++a2) {
        double2* g = G + (size_t)pidx(a, a2) * D;
        k_fro_g<<<f->nblk, BLOCK, 0, s>>>(pdp, a, a2, g);
        count_launch();
        fft_nd<double>(g, pd.n, pd.N, 1, -1, s);
      }
    auto comp = [&](int a, int b) -> int {
      if (kind == QP_COEF_SCALAR) return a == b ? 0 : -1;
      if (kind == QP_COEF_DIAG) return a == b ? a : -1;
      const int lo = std::min(a, b), hi = std::max(a, b);
      return lo * d - lo * (lo - 1) / 2 + (hi - lo);
    };
    for (int b = 0; b < d; ++b)
      for (int b2 = b; b2 < d; ++b2) {
        CK(cudaMemsetAsync(X, 0, D * sizeof(double2), s));
        bool any = false;
        for (int o = 0; o < (b == b2 ? 1 : 2); ++o) {
          const int bb1 = o == 0 ? b : b2, bb2 = o == 0 ? b2 : b;   // (b, b') and, off the diagonal, (b', b)
          for (int a = 0; a < d; ++a)
            for (int a2 = 0; a2 < d; ++a2) {
              const int c1 = comp(a, bb1), c2 = comp(a2, bb2);
              if (c1 < 0 || c2 < 0) continue;
              k_fro_h<<<f->nblk, BLOCK, 0, s>>>(pdp, f->ahat, c1, c2, H);
              count_launch();
              fft_nd<double>(H, pd.n, pd.N, 1, -1, s);
              k_fro_macc<<<f->nblk, BLOCK, 0, s>>>(pd.D, G + (size_t)pidx(a, a2) * D, H, X);
              count_launch();
              any = true;
            }
        }
        if (!any) continue;
        fft_nd<double>(X, pd.n, pd.N, 1, +1, s);
        k_fro_cn<<<f->nblk, BLOCK, 0, s>>>(pdp, b, b2, X, cn);
        count_launch();
      }
    k_fro_final<<<f->nblk, BLOCK, 0, s>>>(pdp, f->ahat, cn, frob, frob32);
    count_launch();
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));
  } catch (...) {
    cudaStreamSynchronize(s);
    for (void* t : tmp) dev_free(t);
    throw;
  }
  for (void* t : tmp) dev_free(t);
}

// ---- apply: gradient -> inverse DFT -> A(y) / D -> DFT -> divergence

// g[b][r] = lambda_b * h[r]
template <typename T>
__global__ void __launch_bounds__(BLOCK) k_grad(const PlanDev* pdp, int nrhs, const cplx<T>* h, cplx<T>* g) {
  const PlanDev& p = *pdp;
  const int D = p.D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    T lk[MAXD];
    int ib[MAXN];
    lambda_of<T>(p, e, lk, ib);
    for (int r = 0; r < nrhs; ++r) {
      const cplx<T> hv = h[(size_t)r * D + e];
      for (int b = 0; b < p.d; ++b) g[((size_t)b * nrhs + r) * D + e] = mk<T>(lk[b] * hv.x, lk[b] * hv.y);
    }
  }
}

// q[a][r] = sum_b (A^{ab}(y) / D) g[b][r], in place
template <typename T>
__global__ void __launch_bounds__(BLOCK) k_coef(const PlanDev* pdp, int nrhs, const T* coef, cplx<T>* g) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d, kind = p.kind;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    T A[MAXD][MAXD];
#pragma unroll
    for (int a = 0; a < MAXD; ++a)
#pragma unroll
      for (int b = 0; b < MAXD; ++b) A[a][b] = (a < d && b < d) ? coef_at<T>(kind, d, coef, D, e, a, b) : T(0);
    for (int r = 0; r < nrhs; ++r) {
      cplx<T> gv[MAXD];
#pragma unroll
      for (int b = 0; b < MAXD; ++b) gv[b] = b < d ? g[((size_t)b * nrhs + r) * D + e] : mk<T>(0, 0);
#pragma unroll
      for (int a = 0; a < MAXD; ++a) {
        if (a < d) {
          cplx<T> q = mk<T>(0, 0);
#pragma unroll
          for (int b = 0; b < MAXD; ++b) {
            q.x = fma(A[a][b], gv[b].x, q.x);
            q.y = fma(A[a][b], gv[b].y, q.y);
          }
          g[((size_t)a * nrhs + r) * D + e] = q;
        }
      }
    }
  }
}

// w[r] = sum_a lambda_a * q[a][r]
template <typename T>
__global__ void __launch_bounds__(BLOCK) k_div(const PlanDev* pdp, int nrhs, const cplx<T>* g, cplx<T>* w) {
  const PlanDev& p = *pdp;
  const int D = p.D;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    T lk[MAXD];
    int ib[MAXN];
    lambda_of<T>(p, e, lk, ib);
    for (int r = 0; r < nrhs; ++r) {
      cplx<T> acc = mk<T>(0, 0);
      for (int a = 0; a < p.d; ++a) {
        const cplx<T> q = g[((size_t)a * nrhs + r) * D + e];
        acc.x = fma(lk[a], q.x, acc.x);
        acc.y = fma(lk[a], q.y, acc.y);
      }
      w[(size_t)r * D + e] = acc;
    }
  }
}

// ---- fused apply: groups of axes transformed in shared-memory tiles
//
// The axes are split into 1 to 3 groups of consecutive axes (each axis <= 32, a group up to all n axes). A pass
// transforms one group of arrays seen as [O][M][I] (M = product of the group's sizes, O of the axes before it,
// I of the axes after): a block stages tiles of L outer x M x R inner elements in shared memory (one padding
// element per 32, so that lines of 8- and 16-byte elements spread over the banks) and runs the register DFT
// along every axis of the group. Tiles divide the arrays exactly. Gradient, coefficient product and
// divergence are applied while the d component tiles of one right-hand side are resident:
//   one group:     [grad, inverse, A(y)/D, forward, divergence]                         one pass
//   two groups:    [grad, inverse G0] [inverse G1, A(y)/D, forward G1] [forward G0, div]   three passes
//   three groups:  as two, with a plain inverse and forward pass over the middle group     five passes
// The DFT is separable, so transforming the groups in this order is the same n-dim transform. Global loads
// and stores of a tile are unrolled so that each thread has all of its elements in flight at once.

constexpr int GP_EPT = 32;   // most tile elements per thread (TS <= GP_EPT * BLOCK)
template <typename T> __host__ __device__ constexpr int GP_BATCH() { return sizeof(T) == 8 ? 8 : 16; }   // loads in flight

__device__ __forceinline__ int tphys(int i) { return i + (i >> 5); }
__device__ __forceinline__ int fdivi(int x, const FastDiv& f) { return (int)fdiv((uint32_t)x, f); }

// One group axis: its stride in the group position, the positions above it, and their fast divisions.
struct AxisLines {
  int sg, nhi;
  FastDiv fsg, fnhi;
};

// DFT of size N along one group axis of ntile tiles (tstride elements apart): lines (l, other group digits, r)
// spread over the block, neighbouring threads on neighbouring r and lower group digits.
template <typename T, int N>
__device__ __noinline__ void tile_axis(cplx<T>* tiles, int ntile, int tstride, const GroupPass& gp, AxisLines ax,
                                       int sign) {
  const int R = gp.R, M = gp.M;
  const int per = gp.L * ax.nhi * ax.sg * R;
  const int step = ax.sg * R;
  for (int job = threadIdx.x; job < per * ntile; job += BLOCK) {
    const int tl = ntile == 1 ? 0 : job / per;
    const int line = job - tl * per;
    int q = fdivi(line, gp.fR);
    const int r = line - q * R;
    int q2 = fdivi(q, ax.fsg);
    const int lo = q - q2 * ax.sg;
    const int l = fdivi(q2, ax.fnhi);
    const int hi = q2 - l * ax.nhi;
    const int base = (l * M + hi * N * ax.sg + lo) * R + r;
    cplx<T>* tp = tiles + (size_t)tl * tstride;
    cplx<T> x[N];
    if ((step & 31) == 0) {
      // the padding is then linear along the line: one add per element
      cplx<T>* lp = tp + tphys(base);
      const int stepP = step + (step >> 5);
#pragma unroll
      for (int k = 0; k < N; ++k) x[k] = lp[k * stepP];
      RegDft<T, N>::run(x, sign);
#pragma unroll
      for (int k = 0; k < N; ++k) lp[k * stepP] = x[k];
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) x[k] = tp[tphys(base + k * step)];
      RegDft<T, N>::run(x, sign);
#pragma unroll
      for (int k = 0; k < N; ++k) tp[tphys(base + k * step)] = x[k];
    }
  }
}

// Every axis of the group, on ntile tiles; ends with a block barrier. (One call site per DFT size keeps the
// kernel's code small.)
template <typename T>
__device__ void tile_transform(cplx<T>* tiles, int ntile, int tstride, const GroupPass& gp, int sign) {
  for (int t = 0; t < gp.ng; ++t) {
    int Nt = 0;
    AxisLines ax;
    switch (t) {
#define QP_AX(i) \
  case i: Nt = gp.Ng[i]; ax = AxisLines{gp.sg[i], gp.nhi[i], gp.fsg[i], gp.fnhi[i]}; break;
      QP_AX(0) QP_AX(1) QP_AX(2) QP_AX(3) QP_AX(4) default: QP_AX(5)
#undef QP_AX
    }
    switch (Nt) {
      case 2: tile_axis<T, 2>(tiles, ntile, tstride, gp, ax, sign); break;
      case 3: tile_axis<T, 3>(tiles, ntile, tstride, gp, ax, sign); break;
      case 4: tile_axis<T, 4>(tiles, ntile, tstride, gp, ax, sign); break;
      case 6: tile_axis<T, 6>(tiles, ntile, tstride, gp, ax, sign); break;
      case 8: tile_axis<T, 8>(tiles, ntile, tstride, gp, ax, sign); break;
      case 9: tile_axis<T, 9>(tiles, ntile, tstride, gp, ax, sign); break;
      case 12: tile_axis<T, 12>(tiles, ntile, tstride, gp, ax, sign); break;
      case 16: tile_axis<T, 16>(tiles, ntile, tstride, gp, ax, sign); break;
      case 18: tile_axis<T, 18>(tiles, ntile, tstride, gp, ax, sign); break;
      case 24: tile_axis<T, 24>(tiles, ntile, tstride, gp, ax, sign); break;
      case 27: tile_axis<T, 27>(tiles, ntile, tstride, gp, ax, sign); break;
      default: tile_axis<T, 32>(tiles, ntile, tstride, gp, ax, sign); break;
    }
    __syncthreads();
  }
}

// lambda_a at the linear mode index e from per-axis tables tab[j][digit][a] = P_aj * k(digit).
template <typename T>
__device__ __forceinline__ void lam_tab(const PlanDev& p, const T* tab, int e, T (&lk)[MAXD]) {
#pragma unroll
  for (int a = 0; a < MAXD; ++a) lk[a] = T(0);
  uint32_t x = (uint32_t)e;
#pragma unroll
  for (int j = MAXN - 1; j >= 0; --j) {
    if (j < p.n) {
      const uint32_t q = fdiv(x, p.div[j]);
      const int dg = (int)(x - q * (uint32_t)p.N[j]);
      x = q;
#pragma unroll
      for (int a = 0; a < MAXD; ++a) lk[a] += tab[(j * 32 + dg) * MAXD + a];
    }
  }
}

// One pass of the fused apply. blockIdx.x: tile (outer-major); blockIdx.y: right-hand side (GP_PLAIN: field).
// Fields g are [d][nrhs][D]; h and w are [nrhs][D]; coef is A^{c}(y) / D, [ncomp][D].
template <typename T, int MODE>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 8 ? 1 : 2) k_fft_group(const PlanDev* pdp, GroupPass gp, int nrhs,
                                                     const cplx<T>* h, cplx<T>* g, cplx<T>* w, const T* coef) {
  __shared__ __align__(16) PlanDev sp;
  __shared__ T tab[MAXN * 32 * MAXD];
  extern __shared__ __align__(16) unsigned char smraw[];
  {
    const int4* src = reinterpret_cast<const int4*>(pdp);
    int4* dst = reinterpret_cast<int4*>(&sp);
    for (int i = threadIdx.x; i < (int)(sizeof(PlanDev) / sizeof(int4)); i += BLOCK) dst[i] = src[i];
  }
  __syncthreads();
  constexpr bool LAM = (MODE == GP_GRAD_INV || MODE == GP_FWD_DIV || MODE == GP_SINGLE);
  if (LAM) {
    for (int i = threadIdx.x; i < MAXN * 32 * MAXD; i += BLOCK) {
      const int a = i % MAXD, dg = (i / MAXD) % 32, j = i / (MAXD * 32);
      T v = T(0);
      if (j < sp.n && a < sp.d && dg < sp.N[j]) {
        const int k = (2 * dg < sp.N[j]) ? dg : dg - sp.N[j];
        v = (T)(pcoef<T>(sp, a, j) * (T)k);
      }
      tab[i] = v;
    }
    __syncthreads();
  }
  cplx<T>* tiles = reinterpret_cast<cplx<T>*>(smraw);
  const int D = sp.D, d = sp.d, kind = sp.kind;
  const int TS = gp.TS;
  const int TSP = tphys(TS - 1) + 1;
  const int to = blockIdx.x / gp.tiles_i, ti = blockIdx.x - to * gp.tiles_i;
  const int base_o = to * gp.L, i0 = ti * gp.R;
  const int y = blockIdx.y;
  // linear index in the array of tile element idx = (l M + pos) R + r: ((base_o + l) M + pos) I + i0 + r, where
  // l M + pos is idx / R itself
  auto lin = [&](int idx) -> int {
    const int q = fdivi(idx, gp.fR);
    const int r = idx - q * gp.R;
    return (base_o * gp.M + q) * gp.I + i0 + r;
  };
  // the index of this thread's u-th element (idx = threadIdx.x + u BLOCK); the one-group pass keeps the division
  // (its registers are taken by the whole transform)
  constexpr bool WALK = MODE != GP_SINGLE;
  const int lin0 = WALK ? lin(threadIdx.x) : 0;
  auto lin_u = [&](int u, int idx) -> int { return (WALK && gp.aff) ? lin0 + u * gp.dlin : lin(idx); };
  const int ntile = (MODE == GP_PLAIN) ? 1 : d;

  // ---- load the tiles: lambda_b h (gradient) or the stored fields, GP_BATCH loads in flight per thread
  constexpr int NB = GP_BATCH<T>();
  if (MODE == GP_GRAD_INV || MODE == GP_SINGLE) {
    for (int u0 = 0; u0 * BLOCK < TS; u0 += NB) {
      cplx<T> hv[NB];
      int ev[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        ev[u] = idx < TS ? lin_u(u0 + u, idx) : 0;
        if (idx < TS) hv[u] = h[(size_t)y * D + ev[u]];
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        if (idx < TS) {
          T lk[MAXD];
          lam_tab<T>(sp, tab, ev[u], lk);
#pragma unroll
          for (int b = 0; b < MAXD; ++b)
            if (b < d) tiles[(size_t)b * TSP + tphys(idx)] = mk<T>(lk[b] * hv[u].x, lk[b] * hv[u].y);
        }
      }
    }
  } else {
    // all tiles of an element from one index computation; NB / 2 elements of every tile in flight
    constexpr int NE = NB / 2;
    const cplx<T>* src0 = g + (size_t)y * D;   // field y (GP_PLAIN) or component 0 of right-hand side y
    const size_t fstride = (size_t)nrhs * D;   // between the component fields of one right-hand side
    for (int u0 = 0; u0 * BLOCK < TS; u0 += NE) {
      cplx<T> v[NE][MAXD];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        if (idx < TS) {
          const int e = lin_u(u0 + u, idx);
#pragma unroll
          for (int b = 0; b < MAXD; ++b)
            if (b < ntile) v[u][b] = src0[(size_t)b * fstride + e];
        }
      }
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        if (idx < TS) {
#pragma unroll
          for (int b = 0; b < MAXD; ++b)
            if (b < ntile) tiles[(size_t)b * TSP + tphys(idx)] = v[u][b];
        }
      }
    }
  }
  __syncthreads();

  // ---- transforms and the coefficient product
  if (MODE == GP_INV_COEF_FWD || MODE == GP_SINGLE) {
    tile_transform<T>(tiles, d, TSP, gp, +1);
    // q_a = sum_b A^{ab}(y) / D g_b at every grid node of the tile (coefficient loads batched)
    const int nc = sp.ncomp;
    constexpr int CB = 4;
    for (int u0 = 0; u0 * BLOCK < TS; u0 += CB) {
      T cv[CB][MAXC];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        const int e = idx < TS ? lin_u(u0 + u, idx) : 0;
#pragma unroll
        for (int c = 0; c < MAXC; ++c) cv[u][c] = (idx < TS && c < nc) ? coef[(size_t)c * D + e] : T(0);
      }
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int idx = threadIdx.x + (u0 + u) * BLOCK;
        if (idx >= TS) break;
        T A[MAXD][MAXD];
        fill_matrix<T>(kind, d, cv[u], A);
        cplx<T> gv[MAXD];
#pragma unroll
        for (int b = 0; b < MAXD; ++b) gv[b] = b < d ? tiles[(size_t)b * TSP + tphys(idx)] : mk<T>(0, 0);
#pragma unroll
        for (int a = 0; a < MAXD; ++a) {
          if (a < d) {
            cplx<T> q = mk<T>(0, 0);
#pragma unroll
            for (int b = 0; b < MAXD; ++b) {
              q.x = fma(A[a][b], gv[b].x, q.x);
              q.y = fma(A[a][b], gv[b].y, q.y);
            }
            tiles[(size_t)a * TSP + tphys(idx)] = q;
          }
        }
      }
    }
    __syncthreads();
    tile_transform<T>(tiles, d, TSP, gp, -1);
  } else {
    tile_transform<T>(tiles, ntile, TSP, gp, MODE == GP_GRAD_INV ? +1 : (MODE == GP_FWD_DIV ? -1 : gp.sign));
  }

  // ---- store: divergence sum_a lambda_a q_a, or the fields
  if (MODE == GP_FWD_DIV || MODE == GP_SINGLE) {
#pragma unroll 4
    for (int u = 0; u < GP_EPT; ++u) {
      const int idx = threadIdx.x + u * BLOCK;
      if (idx >= TS) break;
      const int e = lin_u(u, idx);
      T lk[MAXD];
      lam_tab<T>(sp, tab, e, lk);
      cplx<T> acc = mk<T>(0, 0);
#pragma unroll
      for (int a = 0; a < MAXD; ++a) {
        if (a < d) {
          const cplx<T> q = tiles[(size_t)a * TSP + tphys(idx)];
          acc.x = fma(lk[a], q.x, acc.x);
          acc.y = fma(lk[a], q.y, acc.y);
        }
      }
      w[(size_t)y * D + e] = acc;
    }
  } else {
    cplx<T>* dst0 = g + (size_t)y * D;
    const size_t fstride = (size_t)nrhs * D;
#pragma unroll 4
    for (int u = 0; u < GP_EPT; ++u) {
      const int idx = threadIdx.x + u * BLOCK;
      if (idx >= TS) break;
      const int e = lin_u(u, idx);
#pragma unroll
      for (int b = 0; b < MAXD; ++b)
        if (b < ntile) dst0[(size_t)b * fstride + e] = tiles[(size_t)b * TSP + tphys(idx)];
    }
  }
}

// Largest divisor of x that is <= cap (>= 1).
static long long largest_divisor_le(long long x, long long cap) {
  for (long long v = std::min(x, std::max(1ll, cap)); v > 1; --v)
    if (x % v == 0) return v;
  return 1;
}

// Elements per tile that a pass may stage: ntile tiles (with padding) in about kb KB of shared memory (100 KB:
// two blocks per SM), and at most GP_EPT elements per thread.
static int tile_budget(int esize, int ntile, int kb) {
  const int by_smem = (kb * 1024) / (esize * ntile) * 32 / 33 - 1;
  return std::min(by_smem, GP_EPT * BLOCK);
}

static bool make_pass(const PlanDev& pd, int j0, int ng, int mode, int sign, int esize, int kb, GroupPass& gp) {
  gp = GroupPass();
  if (ng < 1 || ng > MAXN || j0 + ng > pd.n) return false;
  gp.mode = mode;
  gp.sign = sign;
  gp.ng = ng;
  gp.j0 = j0;
  gp.ntile = (mode == GP_PLAIN) ? 1 : std::max(1, pd.d);
  long long M = 1, O = 1, I = 1;
  for (int t = 0; t < ng; ++t) {
    gp.Ng[t] = pd.N[j0 + t];
    if (gp.Ng[t] > 32) return false;
    M *= gp.Ng[t];
  }
  for (int t = ng - 1, st = 1; t >= 0; --t) {
    gp.sg[t] = st;
    st *= gp.Ng[t];
  }
  for (int t = 0; t < ng; ++t) gp.nhi[t] = (int)(M / (gp.Ng[t] * gp.sg[t]));
  for (int j = 0; j < j0; ++j) O *= pd.N[j];
  for (int j = j0 + ng; j < pd.n; ++j) I *= pd.N[j];
  const int budget = tile_budget(esize, gp.ntile, kb);
  if (M > budget) return false;
  gp.M = (int)M;
  gp.O = O;
  gp.I = (int)I;
  if (I > 1) {
    gp.R = (int)largest_divisor_le(I, budget / M);
    gp.L = gp.R == I ? (int)largest_divisor_le(O, budget / (M * I)) : 1;
  } else {
    gp.R = 1;
    gp.L = (int)largest_divisor_le(O, budget / M);
  }
  gp.TS = gp.L * gp.M * gp.R;
  gp.fR = make_fastdiv((uint32_t)gp.R);
  for (int t = 0; t < ng; ++t) {
    gp.fsg[t] = make_fastdiv((uint32_t)gp.sg[t]);
    gp.fnhi[t] = make_fastdiv((uint32_t)gp.nhi[t]);
  }
  gp.tiles_i = (int)(I / gp.R);
  gp.tiles_o = (int)(O / gp.L);
  // the array index of tile element idx is (idx / R) I + idx % R plus the tile's offset, so a step of BLOCK
  // elements is a constant (BLOCK / R) I whenever R divides BLOCK
  gp.aff = (gp.TS > BLOCK && BLOCK % gp.R == 0) ? 1 : 0;
  gp.dlin = gp.aff ? (BLOCK / gp.R) * gp.I : 0;
  gp.smem = (size_t)((gp.TS - 1) + ((gp.TS - 1) >> 5) + 1) * esize * gp.ntile;
  return (long long)gp.tiles_o * gp.tiles_i < (1ll << 31);
}

// Groups of consecutive axes and the passes over them (see above); ok = false leaves the per-axis path.
static FusedSchedule plan_fused(const PlanDev& pd, int esize, int kb) {
  FusedSchedule fs;
  fs.kb = kb;
  const int n = pd.n;
  for (int j = 0; j < n; ++j)
    if (pd.N[j] > 32) return fs;
  GroupPass a, b, c, m1, m2;
  if (make_pass(pd, 0, n, GP_SINGLE, 0, esize, kb, a)) {
    fs.pass[0] = a;
    fs.npass = 1;
    fs.ok = true;
    return fs;
  }
  // two groups [0, s) and [s, n): the most balanced feasible split
  int best = -1;
  long long best_max = 0;
  for (int s = 1; s < n; ++s) {
    if (!make_pass(pd, 0, s, GP_GRAD_INV, 0, esize, kb, a) ||
        !make_pass(pd, s, n - s, GP_INV_COEF_FWD, 0, esize, kb, b))
      continue;
    const long long mx = std::max(a.M, b.M);
    if (best < 0 || mx < best_max) {
      best = s;
      best_max = mx;
    }
  }
  if (best > 0) {
    make_pass(pd, 0, best, GP_GRAD_INV, 0, esize, kb, a);
    make_pass(pd, best, n - best, GP_INV_COEF_FWD, 0, esize, kb, b);
    make_pass(pd, 0, best, GP_FWD_DIV, 0, esize, kb, c);
    fs.pass[0] = a;
    fs.pass[1] = b;
    fs.pass[2] = c;
    fs.npass = 3;
    fs.ok = true;
    return fs;
  }
  // three groups [0, s1), [s1, s2), [s2, n)
  int b1 = -1, b2 = -1;
  for (int s1 = 1; s1 < n - 1; ++s1)
    for (int s2 = s1 + 1; s2 < n; ++s2) {
      if (!make_pass(pd, 0, s1, GP_GRAD_INV, 0, esize, kb, a) ||
          !make_pass(pd, s1, s2 - s1, GP_PLAIN, 1, esize, kb, m1) ||
          !make_pass(pd, s2, n - s2, GP_INV_COEF_FWD, 0, esize, kb, b))
        continue;
      const long long mx = std::max<long long>(std::max(a.M, m1.M), b.M);
      if (b1 < 0 || mx < best_max) {
        b1 = s1;
        b2 = s2;
        best_max = mx;
      }
    }
  if (b1 < 0) return fs;
  make_pass(pd, 0, b1, GP_GRAD_INV, 0, esize, kb, a);
  make_pass(pd, b1, b2 - b1, GP_PLAIN, +1, esize, kb, m1);
  make_pass(pd, b2, n - b2, GP_INV_COEF_FWD, 0, esize, kb, b);
  make_pass(pd, b1, b2 - b1, GP_PLAIN, -1, esize, kb, m2);
  make_pass(pd, 0, b1, GP_FWD_DIV, 0, esize, kb, c);
  fs.pass[0] = a;
  fs.pass[1] = m1;
  fs.pass[2] = b;
  fs.pass[3] = m2;
  fs.pass[4] = c;
  fs.npass = 5;
  fs.ok = true;
  return fs;
}

// Every schedule the group passes can run: one group, every split into two and into three groups of
// consecutive axes, each sized for tile budgets of 48, 100 and 200 KB; distinct by the passes' geometry, in a
// fixed order, followed by the per-axis path (ok = false). The autotuner times them all.
static std::vector<FusedSchedule> fused_candidates(const PlanDev& pd, int esize) {
  std::vector<FusedSchedule> out;
  std::vector<std::string> seen;
  auto add = [&](const FusedSchedule& fs) {
    std::string key = std::to_string(fs.npass);
    for (int i = 0; i < fs.npass; ++i) {
      const GroupPass& g = fs.pass[i];
      key += ":" + std::to_string(g.j0) + "," + std::to_string(g.ng) + "," + std::to_string(g.mode) + "," +
             std::to_string(g.L) + "," + std::to_string(g.R);
    }
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) return;
    seen.push_back(key);
    out.push_back(fs);
  };
  const int n = pd.n;
  bool small = true;
  for (int j = 0; j < n; ++j) small = small && pd.N[j] <= 32;
  const int budgets[3] = {48, 100, 200};
  for (int bi = 0; bi < 3 && small; ++bi) {
    const int kb = budgets[bi];
    FusedSchedule fs;
    fs.ok = true;
    fs.kb = kb;
    GroupPass a, b, c, m1, m2;
    if (make_pass(pd, 0, n, GP_SINGLE, 0, esize, kb, a)) {
      fs.pass[0] = a;
      fs.npass = 1;
      add(fs);
    }
    for (int s1 = 1; s1 < n; ++s1) {
      if (make_pass(pd, 0, s1, GP_GRAD_INV, 0, esize, kb, a) &&
          make_pass(pd, s1, n - s1, GP_INV_COEF_FWD, 0, esize, kb, b) &&
          make_pass(pd, 0, s1, GP_FWD_DIV, 0, esize, kb, c)) {
        fs.pass[0] = a;
        fs.pass[1] = b;
        fs.pass[2] = c;
        fs.npass = 3;
        add(fs);
      }
    }
    for (int s1 = 1; s1 < n - 1; ++s1)
      for (int s2 = s1 + 1; s2 < n; ++s2) {
        if (make_pass(pd, 0, s1, GP_GRAD_INV, 0, esize, kb, a) &&
            make_pass(pd, s1, s2 - s1, GP_PLAIN, +1, esize, kb, m1) &&
            make_pass(pd, s2, n - s2, GP_INV_COEF_FWD, 0, esize, kb, b) &&
            make_pass(pd, s1, s2 - s1, GP_PLAIN, -1, esize, kb, m2) &&
            make_pass(pd, 0, s1, GP_FWD_DIV, 0, esize, kb, c)) {
          fs.pass[0] = a;
          fs.pass[1] = m1;
          fs.pass[2] = b;
          fs.pass[3] = m2;
          fs.pass[4] = c;
          fs.npass = 5;
          add(fs);
        }
      }
  }
  out.push_back(FusedSchedule());   // the per-axis path
  return out;
}

static std::string schedule_text(const FusedSchedule& fs) {
  if (!fs.ok) return "per-axis passes";
  std::string t;
  for (int i = 0; i < fs.npass; ++i) {
    const GroupPass& g = fs.pass[i];
    if (g.mode == GP_FWD_DIV || (g.mode == GP_PLAIN && g.sign < 0)) continue;   // mirrors of earlier passes
    t += "[" + std::to_string(g.j0) + "," + std::to_string(g.j0 + g.ng) + ")";
  }
  const GroupPass& g0 = fs.pass[0];
  return "axis groups " + t + ", " + std::to_string(fs.npass) + " passes, tile budget " + std::to_string(fs.kb) +
         " KB (first pass: tiles of " + std::to_string(g0.L) + " x " + std::to_string(g0.M) + " x " +
         std::to_string(g0.R) + ")";
}

template <typename T, int MODE>
static void launch_group(const GroupPass& gp, const PlanDev* pdp, int nrhs, int ny, const cplx<T>* h, cplx<T>* g,
                         cplx<T>* w, const T* coef, cudaStream_t s) {
  auto fn = k_fft_group<T, MODE>;
  // the 48 KB default covers static + dynamic shared memory (about 7 KB static here): opt in above 40 KB
  if (gp.smem > 40 * 1024) CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gp.smem));
  dim3 grid((unsigned)((long long)gp.tiles_o * gp.tiles_i), (unsigned)ny);
  fn<<<grid, BLOCK, gp.smem, s>>>(pdp, gp, nrhs, h, g, w, coef);
  count_launch();
}

template <typename T>
static void run_fused(const FusedSchedule& fs, const PlanDev& pd, const PlanDev* pdp, const cplx<T>* h, cplx<T>* g,
                      cplx<T>* w, const T* coef, int nrhs, cudaStream_t s) {
  for (int i = 0; i < fs.npass; ++i) {
    const GroupPass& gp = fs.pass[i];
    switch (gp.mode) {
      case GP_SINGLE: launch_group<T, GP_SINGLE>(gp, pdp, nrhs, nrhs, h, g, w, coef, s); break;
      case GP_GRAD_INV: launch_group<T, GP_GRAD_INV>(gp, pdp, nrhs, nrhs, h, g, w, coef, s); break;
      case GP_INV_COEF_FWD: launch_group<T, GP_INV_COEF_FWD>(gp, pdp, nrhs, nrhs, h, g, w, coef, s); break;
      case GP_FWD_DIV: launch_group<T, GP_FWD_DIV>(gp, pdp, nrhs, nrhs, h, g, w, coef, s); break;
      default: launch_group<T, GP_PLAIN>(gp, pdp, nrhs, pd.d * nrhs, h, g, w, coef, s); break;
    }
  }
}

template <typename T> static cplx<T>* fields_of(FftPlan* f);
template <> double2* fields_of<double>(FftPlan* f) { return f->f64; }
template <> float2* fields_of<float>(FftPlan* f) { return f->f32; }
template <typename T> static const T* coef_of(FftPlan* f);
template <> const double* coef_of<double>(FftPlan* f) { return f->coef64; }
template <> const float* coef_of<float>(FftPlan* f) { return f->coef32; }

// The per-axis path: gradient, n-dim inverse FFT of the d fields, coefficient product, forward FFT, divergence.
template <typename T>
static void run_axis(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const cplx<T>* h, cplx<T>* w, int nrhs,
                     cudaStream_t s) {
  cplx<T>* g = fields_of<T>(f);
  k_grad<T><<<f->nblk, BLOCK, 0, s>>>(pdp, nrhs, h, g);
  count_launch();
  fft_nd<T>(g, pd.n, pd.N, (long long)pd.d * nrhs, +1, s);
  k_coef<T><<<f->nblk, BLOCK, 0, s>>>(pdp, nrhs, coef_of<T>(f), g);
  count_launch();
  fft_nd<T>(g, pd.n, pd.N, (long long)pd.d * nrhs, -1, s);
  k_div<T><<<f->nblk, BLOCK, 0, s>>>(pdp, nrhs, g, w);
  count_launch();
}

template <typename T>
void fft_apply(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, const cplx<T>* h, cplx<T>* w, int nrhs,
               cudaStream_t s) {
  cplx<T>* g = fields_of<T>(f);
  if (!g || nrhs > f->max_rhs)
    raise(QP_ERR_INVALID_ARG, "FFT plan has no workspace for this precision / number of right-hand sides");
  const FusedSchedule& fs = (sizeof(T) == 8) ? f->fused64 : f->fused32;
  if (fs.ok) run_fused<T>(fs, pd, pdp, h, g, w, coef_of<T>(f), nrhs, s);
  else run_axis<T>(f, pd, pdp, h, w, nrhs, s);
  CK_LAUNCH();
}

// ---- autotuner of the apply schedule

namespace {
std::mutex g_tune_mu;
// geometry and precision -> chosen candidate and every candidate's timing (ms per apply), so that a plan served
// from the cache reports the same schedule and timings as the plan that was timed
std::map<std::string, std::pair<int, std::vector<float>>> g_tune_cache;
std::atomic<int> g_autotune{1};
}  // namespace

void fft_set_autotune(bool on) { g_autotune.store(on ? 1 : 0); }
bool fft_autotune_on() { return g_autotune.load() != 0; }

template <typename T>
static void tune_precision(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, cudaStream_t s) {
  ScheduleSet& ss = sizeof(T) == 8 ? f->sched64 : f->sched32;
  FusedSchedule& use = sizeof(T) == 8 ? f->fused64 : f->fused32;
  if (!fields_of<T>(f) || ss.cand.empty()) return;
  std::string key = std::to_string(sizeof(T)) + "/" + std::to_string(pd.d) + "/" + std::to_string(pd.kind) + "/" +
                    std::to_string(f->max_rhs);
  for (int j = 0; j < pd.n; ++j) key += "/" + std::to_string(pd.N[j]);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && it->second.first < (int)ss.cand.size() &&
        it->second.second.size() == ss.cand.size()) {
      ss.chosen = it->second.first;
      ss.ms = it->second.second;
      use = ss.cand[ss.chosen];
      return;
    }
  }
  if (!g_autotune.load()) return;   // keep the balanced-split heuristic
  const int nr = f->max_rhs;
  const size_t bytes = (size_t)nr * pd.D * sizeof(cplx<T>);
  cplx<T>* h = static_cast<cplx<T>*>(dev_alloc(bytes, s));
  cplx<T>* w = static_cast<cplx<T>*>(dev_alloc(bytes, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ss.ms.assign(ss.cand.size(), INFINITY);
  try {
    CK(cudaMemsetAsync(h, 0, bytes, s));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (size_t i = 0; i < ss.cand.size(); ++i) {
      const FusedSchedule& fs = ss.cand[i];
      auto run = [&]() {
        if (fs.ok) run_fused<T>(fs, pd, pdp, h, fields_of<T>(f), w, coef_of<T>(f), nr, s);
        else run_axis<T>(f, pd, pdp, h, w, nr, s);
      };
      try {
        run();   // warm-up (and the shared-memory opt-in of its kernels)
        CK(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) run();
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK_LAUNCH();
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ss.ms[i] = ms / 3.f;
      } catch (const QpError&) {
        // a configuration this device refuses (launch error, nothing ran): not a candidate here
        if (cudaStreamSynchronize(s) != cudaSuccess) throw;
        cudaGetLastError();
      }
    }
  } catch (...) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    dev_free(h);
    dev_free(w);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaStreamSynchronize(s));
  dev_free(h);
  dev_free(w);
  int best = 0;
  for (size_t i = 1; i < ss.ms.size(); ++i)
    if (ss.ms[i] < ss.ms[best]) best = (int)i;
  ss.chosen = best;
  use = ss.cand[best];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best, ss.ms};
}

// The tuning cache in a text file, for later processes on the same kind of GPU: a header line with the format
// version and the device name, then one line per entry: key, chosen candidate, candidate count, their timings.
static std::string device_name() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  std::string name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  return name;
}

int fft_tune_cache_save(const char* path) {
  const std::string dev = device_name();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* fp = std::fopen(path, "w");
  if (!fp) return -1;
  std::fprintf(fp, "qp-fft-tune-cache 1 %s\n", dev.c_str());
  int n = 0;
  for (const auto& kv : g_tune_cache) {
    std::fprintf(fp, "%s %d %zu", kv.first.c_str(), kv.second.first, kv.second.second.size());
    for (float ms : kv.second.second) std::fprintf(fp, " %.9g", (double)ms);
    std::fprintf(fp, "\n");
    ++n;
  }
  const bool ok = std::fclose(fp) == 0;
  return ok ? n : -1;
}

int fft_tune_cache_load(const char* path) {
  const std::string dev = device_name();
  FILE* fp = std::fopen(path, "r");
  if (!fp) return -1;
  std::vector<std::pair<std::string, std::pair<int, std::vector<float>>>> entries;
  char head[64] = {}, name[256] = {};
  int version = 0;
  bool ok = std::fscanf(fp, "%63s %d %255s", head, &version, name) == 3 && std::string(head) == "qp-fft-tune-cache" &&
            version == 1;
  if (ok && dev != name) {
    std::fclose(fp);
    return -2;   // timed on another kind of GPU
  }
  while (ok) {
    char key[256] = {};
    int chosen = 0;
    unsigned long cnt = 0;
    const int got = std::fscanf(fp, "%255s %d %lu", key, &chosen, &cnt);
    if (got == EOF) break;
    if (got != 3 || cnt > 100000 || chosen < 0 || (unsigned long)chosen >= cnt) {
      ok = false;
      break;
    }
    std::vector<float> ms(cnt);
    for (unsigned long i = 0; ok && i < cnt; ++i) ok = std::fscanf(fp, "%f", &ms[i]) == 1;
    if (ok) entries.push_back({key, {chosen, ms}});
  }
  std::fclose(fp);
  if (!ok) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : entries) g_tune_cache[e.first] = e.second;
  return (int)entries.size();
}

void fft_tune_cache_clear() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

void fft_autotune(FftPlan* f, const PlanDev& pd, const PlanDev* pdp, cudaStream_t s) {
  if (f->precisions & 1) tune_precision<double>(f, pd, pdp, s);
  if (f->precisions & 2) tune_precision<float>(f, pd, pdp, s);
}

int fft_schedule_count(const FftPlan* f, bool fp64) { return (int)(fp64 ? f->sched64 : f->sched32).cand.size(); }

int fft_schedule_get(const FftPlan* f, bool fp64, std::string& text, float& ms) {
  const ScheduleSet& ss = fp64 ? f->sched64 : f->sched32;
  const FusedSchedule& use = fp64 ? f->fused64 : f->fused32;
  text = schedule_text(use);
  ms = (ss.chosen >= 0 && ss.chosen < (int)ss.ms.size()) ? ss.ms[ss.chosen] : -1.f;
  return ss.chosen;
}

void fft_schedule_set(FftPlan* f, bool fp64, int index) {
  ScheduleSet& ss = fp64 ? f->sched64 : f->sched32;
  if (index < 0 || index >= (int)ss.cand.size()) raise(QP_ERR_INVALID_ARG, "schedule index out of range");
  ss.chosen = index;
  (fp64 ? f->fused64 : f->fused32) = ss.cand[index];
}
template void fft_apply<double>(FftPlan*, const PlanDev&, const PlanDev*, const double2*, double2*, int, cudaStream_t);
template void fft_apply<float>(FftPlan*, const PlanDev&, const PlanDev*, const float2*, float2*, int, cudaStream_t);

// F_j(k) = i sum_a lambda_a(k) A~^{aj}_k, F_j(0) = 0
__global__ void __launch_bounds__(BLOCK) k_rhs_fft(const PlanDev* pdp, const double2* ahat, int j0, int nrhs,
                                                   double2* F) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    for (int jj = 0; jj < nrhs; ++jj) {
      const int j = j0 + jj;
      double2 z = make_double2(0.0, 0.0);
      for (int a = 0; a < d; ++a) {
        int comp = -1;
        if (p.kind == QP_COEF_SCALAR) comp = a == j ? 0 : -1;
        else if (p.kind == QP_COEF_DIAG) comp = a == j ? a : -1;
        else comp = sym_idx(a, j, d);
        if (comp < 0) continue;
        const double2 c = ahat[(size_t)comp * D + e];
        z.x += lk[a] * c.x;
        z.y += lk[a] * c.y;
      }
      F[(size_t)jj * D + e] = e == 0 ? make_double2(0.0, 0.0) : make_double2(-z.y, z.x);
    }
  }
}

void fft_rhs(FftPlan* f, const PlanDev&, const PlanDev* pdp, int j0, int nrhs, double2* F, cudaStream_t s) {
  k_rhs_fft<<<f->nblk, BLOCK, 0, s>>>(pdp, f->ahat, j0, nrhs, F);
  count_launch();
  CK_LAUNCH();
}

// A*_ij = A~^{ij}_0 + i sum_k sum_b A~^{ib}_{-k} lambda_b(k) U_j(k): block partials, then a fixed-order final sum.
__global__ void __launch_bounds__(BLOCK) k_astar_fft(const PlanDev* pdp, const double2* ahat, const double2* U,
                                                     double* part) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d;
  double v[2 * MAXD * MAXD];
#pragma unroll
  for (int q = 0; q < 2 * MAXD * MAXD; ++q) v[q] = 0.0;
  for (int e = blockIdx.x * BLOCK + threadIdx.x; e < D; e += gridDim.x * BLOCK) {
    double lk[MAXD];
    int ib[MAXN];
    lambda_of<double>(p, e, lk, ib);
    int eneg = 0;   // storage index of -k
    for (int ax = 0; ax < p.n; ++ax) eneg += ((p.N[ax] - ib[ax]) % p.N[ax]) * p.stride[ax];
#pragma unroll
    for (int i = 0; i < MAXD; ++i) {
      if (i >= d) continue;
      double2 s = make_double2(0.0, 0.0);   // sum_b A~^{ib}_{-k} lambda_b(k)
      for (int b = 0; b < d; ++b) {
        int comp = -1;
        if (p.kind == QP_COEF_SCALAR) comp = i == b ? 0 : -1;
        else if (p.kind == QP_COEF_DIAG) comp = i == b ? i : -1;
        else comp = sym_idx(i, b, d);
        if (comp < 0) continue;
        const double2 c = ahat[(size_t)comp * D + eneg];
        s.x += c.x * lk[b];
        s.y += c.y * lk[b];
      }
#pragma unroll
      for (int j = 0; j < MAXD; ++j) {
        if (j >= d) continue;
        const double2 u = U[(size_t)j * D + e];
        const double pr = s.x * u.x - s.y * u.y, pim = s.x * u.y + s.y * u.x;
        v[2 * (i * MAXD + j)] += -pim;
        v[2 * (i * MAXD + j) + 1] += pr;
      }
    }
  }
  block_reduce<2 * MAXD * MAXD>(v);
  if (threadIdx.x == 0)
    for (int q = 0; q < 2 * MAXD * MAXD; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = v[q];
}

__global__ void k_astar_fft_final(const PlanDev* pdp, const double2* ahat, const double* part, int nb, double* out) {
  const PlanDev& p = *pdp;
  const int D = p.D, d = p.d;
  double v[2 * MAXD * MAXD];
#pragma unroll
  for (int q = 0; q < 2 * MAXD * MAXD; ++q) v[q] = 0.0;
  for (int i = threadIdx.x; i < nb; i += BLOCK)
#pragma unroll
    for (int q = 0; q < 2 * MAXD * MAXD; ++q) v[q] += part[(size_t)q * nb + i];
  block_reduce<2 * MAXD * MAXD>(v);
  if (threadIdx.x == 0) {
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        int comp = -1;
        if (p.kind == QP_COEF_SCALAR) comp = i == j ? 0 : -1;
        else if (p.kind == QP_COEF_DIAG) comp = i == j ? i : -1;
        else comp = sym_idx(i, j, d);
        const double2 c0 = comp >= 0 ? ahat[(size_t)comp * D] : make_double2(0.0, 0.0);
        out[2 * (i * d + j)] = c0.x + v[2 * (i * MAXD + j)];
        out[2 * (i * d + j) + 1] = c0.y + v[2 * (i * MAXD + j) + 1];
      }
  }
}

void fft_astar(FftPlan* f, const PlanDev&, const PlanDev* pdp, const double2* U, double* out, cudaStream_t s) {
  k_astar_fft<<<f->nblk, BLOCK, 0, s>>>(pdp, f->ahat, U, f->part);
  k_astar_fft_final<<<1, BLOCK, 0, s>>>(pdp, f->ahat, f->part, f->nblk, out);
  count_launch(2);
  CK_LAUNCH();
}

}  // namespace qp
