// Field-wide kernels around the fixed-point map: the inner products and
// tall-skinny projections of the recursive projection method (Section 3,
// Eqs. 3.10-3.13), the Newton step on the unstable subspace, the strain
// combine of Algorithm 2 and the constitutive law sigma = C(x) : eps.
//
// Fields are [6][n] float32 (components 11 22 33 23 13 12).  The inner
// product is the tensor Frobenius product (weights 1,1,1,2,2,2).  Each
// thread accumulates a bounded number of products in float32; the block and
// grid reductions run in float64 with a fixed order (deterministic).
#include <math.h>

#include <atomic>

#include "rpm_internal.h"

namespace rpm {

constexpr int kRedThreads = 256;
constexpr int kPerThread = 8;        // float4 per thread per dot pass (32 products)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Error-free sum a + b = s + e (Knuth's TwoSum, six float32 operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warp sum of float values as an unevaluated pair hi + lo: every level of the
// shuffle tree is a TwoSum, so the rounding errors of the float32 tree are
// carried exactly in lo (float64 arithmetic is slow on this part; the pair
// gives about 48 significant bits).
__device__ __forceinline__ void warp_sum_compensated(float v, float& hi, float& lo) {
  hi = v;
  lo = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, ohi, s, e);
    hi = s;
    lo = lo + olo + e;
  }
}

// Block-reduce M float values per thread (acc) into partials[row(j) * nblk + blockIdx.x],
// row(0) = 0 when row0 == 0 (skipped otherwise), row(j) = row0 + j for j >= 1.
// Warp level in compensated float32, warps and blocks combined in float64.
template <int M>
__device__ __forceinline__ void block_store(const float* acc, int m, int row0, double* partials,
                                            int nblk) {
  __shared__ double red[kRedThreads / 32][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < M; ++j) {
    if (j < m) {
      float hi, lo;
      warp_sum_compensated(acc[j], hi, lo);
      if (lane == 0) red[warp][j] = (double)hi + (double)lo;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j == 0 && row0 != 0) continue;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) s += red[w][j];
    partials[(size_t)(j == 0 ? 0 : row0 + j) * nblk + blockIdx.x] = s;
  }
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// acc[0] = sum w |x - xm|^2 and acc[1 + j] = sum w (x - xm) . Y_j; without xm,
// sum w |x|^2 and sum w x . Y_j.  The difference is formed per element before
// any product, so Z^T (xi - eps) keeps its accuracy when xi and eps agree to
// many digits (near convergence).
// Partial sums go to rows [0] (the norm) and [1 + row0 + j] of `partials`.
template <int KMAX>
__device__ __forceinline__ void dots_body(const float4* __restrict__ x,
                                          const float4* __restrict__ xm,
                                          const float4* __restrict__ Y, long long ys4, int K,
                                          int row0, long long n4, double* partials, int nblk) {
  // The thread's kPerThread difference vectors stay in registers; each basis
  // vector is then read as kPerThread independent 16-byte loads issued
  // together, and its warp sum is taken at once (no accumulator stays live
  // across the vectors, which keeps the register count at three blocks per SM).
  __shared__ double red[kRedThreads / 32][KMAX + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long total = 6 * n4;
  const long long base = (long long)blockIdx.x * kRedThreads * kPerThread + threadIdx.x;
  float4 d[kPerThread];
  float w[kPerThread];
#pragma unroll
  for (int r = 0; r < kPerThread; ++r) {
    const long long q = base + (long long)r * kRedThreads;
    const bool in = q < total;
    w[r] = in ? ((q >= 3 * n4) ? 2.f : 1.f) : 0.f;
    d[r] = in ? x[q] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (xm) {
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) {
      const long long q = base + (long long)r * kRedThreads;
      if (q < total) {
        const float4 b = xm[q];
        d[r] = make_float4(d[r].x - b.x, d[r].y - b.y, d[r].z - b.z, d[r].w - b.w);
      }
    }
  }
  {
    float a = 0.f, hi, lo;
#pragma unroll
    for (int r = 0; r < kPerThread; ++r) a = fmaf(w[r], dot4(d[r], d[r]), a);
    warp_sum_compensated(a, hi, lo);
    if (lane == 0) red[warp][0] = (double)hi + (double)lo;
  }
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < K) {
      const float4* yj = Y + j * ys4;
      float4 y[kPerThread];
#pragma unroll
      for (int r = 0; r < kPerThread; ++r) {
        const long long q = base + (long long)r * kRedThreads;
        y[r] = q < total ? yj[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float a = 0.f, hi, lo;
#pragma unroll
      for (int r = 0; r < kPerThread; ++r) a = fmaf(w[r], dot4(d[r], y[r]), a);
      warp_sum_compensated(a, hi, lo);
      if (lane == 0) red[warp][1 + j] = (double)hi + (double)lo;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= K; j += blockDim.x) {
    if (j == 0 && row0 != 0) continue;
    double t = 0.0;
#pragma unroll
    for (int v = 0; v < kRedThreads / 32; ++v) t += red[v][j];
    partials[(size_t)(j == 0 ? 0 : row0 + j) * nblk + blockIdx.x] = t;
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kRedThreads, 3) k_dots(const float4* __restrict__ x,
                                                      const float4* __restrict__ xm,
                                                      const float4* __restrict__ Y, long long ys4,
                                                      int K, int row0, long long n4,
                                                      double* partials, int nblk) {
  dots_body<KMAX>(x, xm, Y, ys4, K, row0, n4, partials, nblk);
}

// k_dots (K <= 32) whose last block to finish also adds the per-block rows in
// a fixed order (a warp per row: lanes take every 32nd block, then a fixed
// shuffle tree) into sums[0..K] and, when M is given, takes the Newton step
// of k_newton with p = K.  The ticket counter is zero between launches (the
// last block resets it).  One launch instead of three.
template <int KMAX>
__global__ void __launch_bounds__(kRedThreads, 3) k_dots_fused(
    const float4* __restrict__ x, const float4* __restrict__ xm, const float4* __restrict__ Y,
    long long ys4, int K, long long n4, double* partials, int nblk, double* sums,
    unsigned int* ticket, const double* __restrict__ M, double* c, double* res_out,
    double inv_norm) {
  dots_body<KMAX>(x, xm, Y, ys4, K, 0, n4, partials, nblk);
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j <= K; j += kRedThreads / 32) {
    // 8 independent chains per lane (loads in flight), added in a fixed order
    const double* row = partials + (size_t)j * nblk;
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int b = lane;
    for (; b + 7 * 32 < nblk; b += 8 * 32) {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] += __ldcg(row + b + q * 32);   // L2, not L1
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (b + q * 32 < nblk) v[q] += __ldcg(row + b + q * 32);
    double t = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    t = warp_sum(t);
    if (lane == 0) sums[j] = t;
  }
  __syncthreads();
  if (M) {
    __shared__ double d[32];
    for (int j = threadIdx.x; j < K; j += blockDim.x) d[j] = sums[1 + j];
    __syncthreads();
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      double t = -d[j];
      for (int k = 0; k < K; ++k) t += M[(size_t)j * K + k] * d[k];
      c[j] = t;
    }
    if (threadIdx.x == 0) res_out[0] = sqrt(sums[0]) * inv_norm;   // NaN stays NaN
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

cudaError_t launch_dots_fused(const float* x, const float* x_minus, const float* Y,
                              long long ystride, int K, long long n, double* partials, int nblk,
                              double* sums, unsigned int* ticket, const double* M, double* c,
                              double* res_out, double inv_norm, cudaStream_t st) {
  if (K > 32) return cudaErrorInvalidValue;
  const long long n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* m4 = reinterpret_cast<const float4*>(x_minus);
  const float4* y4 = reinterpret_cast<const float4*>(Y);
  const long long ys4 = ystride / 4;
#define RPM_FUSED(KM)                                                                       \
  k_dots_fused<KM><<<nblk, kRedThreads, 0, st>>>(x4, m4, y4, ys4, K, n4, partials, nblk, sums, \
                                                 ticket, M, c, res_out, inv_norm)
  if (K <= 2)
    RPM_FUSED(2);
  else if (K <= 8)
    RPM_FUSED(8);
  else if (K <= 16)
    RPM_FUSED(16);
  else
    RPM_FUSED(32);
#undef RPM_FUSED
  return cudaGetLastError();
}

int dots_blocks_for(long long n) {
  const long long total = 6 * (n / 4);
  return (int)((total + (long long)kRedThreads * kPerThread - 1) / ((long long)kRedThreads * kPerThread));
}

cudaError_t launch_dots(const float* x, const float* x_minus, const float* Y, long long ystride,
                        int K, long long n, double* partials, int nblk, cudaStream_t st) {
  const long long n4 = n / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* m4 = reinterpret_cast<const float4*>(x_minus);
  const long long ys4 = ystride / 4;
  // K > 32: chunks of 32 basis vectors; the norm row is written by chunk 0
  for (int k0 = 0; k0 == 0 || k0 < K; k0 += 32) {
    const int Kc = K - k0 < 32 ? K - k0 : 32;
    const float4* y4 = reinterpret_cast<const float4*>(Y) + (Y ? k0 * ys4 : 0);
    if (Kc <= 2)
      k_dots<2><<<nblk, kRedThreads, 0, st>>>(x4, m4, y4, ys4, Kc, k0, n4, partials, nblk);
    else if (Kc <= 8)
      k_dots<8><<<nblk, kRedThreads, 0, st>>>(x4, m4, y4, ys4, Kc, k0, n4, partials, nblk);
    else if (Kc <= 16)
      k_dots<16><<<nblk, kRedThreads, 0, st>>>(x4, m4, y4, ys4, Kc, k0, n4, partials, nblk);
    else
      k_dots<32><<<nblk, kRedThreads, 0, st>>>(x4, m4, y4, ys4, Kc, k0, n4, partials, nblk);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int dots_launches(int K) { return K <= 32 ? 1 : (K + 31) / 32; }

// out[j] = sum_b partials[j * nblk + b], one block per j, fixed order.
__global__ void __launch_bounds__(kRedThreads) k_reduce(const double* __restrict__ partials, int nblk,
                                                        double* out) {
  const int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partials[(size_t)j * nblk + b];
  __shared__ double red[kRedThreads / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) t += red[w];
    out[j] = t;
  }
}

cudaError_t launch_reduce_partials(const double* partials, int nblk, int m, double* out,
                                   cudaStream_t st) {
  k_reduce<<<m, kRedThreads, 0, st>>>(partials, nblk, out);
  return cudaGetLastError();
}

// out = xs * x + sum_j coef[j] * Y_j   (coef in float64 on the device)
// (out may alias x).  The basis vectors are read in groups of 8 so that each
// thread keeps 8 independent 16-byte loads in flight at a modest register count.
template <int KMAX>
__global__ void __launch_bounds__(kRedThreads, 3) k_combine(float4* out, const float4* x, float xs,
                                                            const float4* __restrict__ Y,
                                                            long long ys4, int K,
                                                            const double* __restrict__ coef,
                                                            float cscale, long long total4) {
  __shared__ float cf[KMAX > 0 ? KMAX : 1];
  for (int j = threadIdx.x; j < K; j += blockDim.x) cf[j] = (float)(coef[j] * (double)cscale);
  __syncthreads();
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total4;
       q += (long long)gridDim.x * blockDim.x) {
    float4 a = x ? x[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    a = make_float4(a.x * xs, a.y * xs, a.z * xs, a.w * xs);
#pragma unroll 1
    for (int j0 = 0; j0 < K; j0 += 8) {
      float4 y[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (j0 + u < K) y[u] = Y[(j0 + u) * ys4 + q];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (j0 + u < K) {
          const float c = cf[j0 + u];
          a.x = fmaf(c, y[u].x, a.x);
          a.y = fmaf(c, y[u].y, a.y);
          a.z = fmaf(c, y[u].z, a.z);
          a.w = fmaf(c, y[u].w, a.w);
        }
      }
    }
    out[q] = a;
  }
}

static int stream_blocks(long long total4) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v;
  }
  const long long want = (total4 + kRedThreads - 1) / kRedThreads;
  const long long cap = (long long)sms * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Grid of a grid-stride kernel: the blocks that are resident at once (so no
// partial last wave), at most one block per 256 threads' worth of work.
// (the occupancy query runs once per kernel instance: `slot` caches it)
template <typename Kern>
static int resident_grid(Kern kernel, long long total4, std::atomic<int>& slot) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v;
  }
  int per_sm = slot.load();
  if (per_sm < 1) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRedThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    slot.store(per_sm);
  }
  const long long want = (total4 + kRedThreads - 1) / kRedThreads;
  const long long cap = (long long)sms * per_sm;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

static std::atomic<int> g_combine_occ[4];   // resident blocks per SM of k_combine<2, 8, 16, 32>

cudaError_t launch_combine(float* out, const float* x, float xscale, const float* Y,
                           long long ystride, int K, const double* coef, float cscale,
                           long long n, cudaStream_t st) {
  const long long total4 = 6 * (n / 4);
  float4* o4 = reinterpret_cast<float4*>(out);
  const long long ys4 = ystride / 4;
  // K > 32: the first chunk forms xs * x + ..., later chunks accumulate into out
  for (int k0 = 0; k0 == 0 || k0 < K; k0 += 32) {
    const int Kc = K - k0 < 32 ? K - k0 : 32;
    const float4* x4 = k0 == 0 ? reinterpret_cast<const float4*>(x) : o4;
    const float xs = k0 == 0 ? xscale : 1.f;
    const float4* y4 = reinterpret_cast<const float4*>(Y) + (Y ? k0 * ys4 : 0);
    const double* cf = coef ? coef + k0 : nullptr;
    if (Kc <= 2)
      k_combine<2><<<resident_grid(k_combine<2>, total4, g_combine_occ[0]), kRedThreads, 0, st>>>(
          o4, x4, xs, y4, ys4, Kc, cf, cscale, total4);
    else if (Kc <= 8)
      k_combine<8><<<resident_grid(k_combine<8>, total4, g_combine_occ[1]), kRedThreads, 0, st>>>(
          o4, x4, xs, y4, ys4, Kc, cf, cscale, total4);
    else if (Kc <= 16)
      k_combine<16><<<resident_grid(k_combine<16>, total4, g_combine_occ[2]), kRedThreads, 0, st>>>(
          o4, x4, xs, y4, ys4, Kc, cf, cscale, total4);
    else
      k_combine<32><<<resident_grid(k_combine<32>, total4, g_combine_occ[3]), kRedThreads, 0, st>>>(
          o4, x4, xs, y4, ys4, Kc, cf, cscale, total4);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int combine_launches(int K) { return K <= 32 ? 1 : (K + 31) / 32; }

// sigma = C(x) : eps (Eq. 2.2), optionally stored, and per-component sums.
__global__ void __launch_bounds__(kRedThreads) k_stress(const float4* __restrict__ eps,
                                                        const uchar4* __restrict__ phase,
                                                        const float2* __restrict__ cmat,
                                                        float4* __restrict__ sig, long long n4,
                                                        double* partials, int nblk) {
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const long long base = (long long)blockIdx.x * kRedThreads * kPerThread + threadIdx.x;
#pragma unroll 1
  for (int r = 0; r < kPerThread; ++r) {
    const long long q = base + (long long)r * kRedThreads;
    if (q >= n4) break;
    const uchar4 ph = phase[q];
    const float2 m0 = cmat[ph.x], m1 = cmat[ph.y], m2 = cmat[ph.z], m3 = cmat[ph.w];
    float4 e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps[c * n4 + q];
    const float4 tr = make_float4(e[0].x + e[1].x + e[2].x, e[0].y + e[1].y + e[2].y,
                                  e[0].z + e[1].z + e[2].z, e[0].w + e[1].w + e[2].w);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float4 s = make_float4(2.f * m0.y * e[c].x, 2.f * m1.y * e[c].y, 2.f * m2.y * e[c].z,
                             2.f * m3.y * e[c].w);
      if (c < 3) {
        s.x = fmaf(m0.x, tr.x, s.x);
        s.y = fmaf(m1.x, tr.y, s.y);
        s.z = fmaf(m2.x, tr.z, s.z);
        s.w = fmaf(m3.x, tr.w, s.w);
      }
      if (sig) sig[c * n4 + q] = s;
      acc[c] += (s.x + s.y) + (s.z + s.w);
    }
  }
  block_store<6>(acc, 6, 0, partials, nblk);
}

int stress_blocks_for(long long n) {
  const long long n4 = n / 4;
  return (int)((n4 + (long long)kRedThreads * kPerThread - 1) / ((long long)kRedThreads * kPerThread));
}

cudaError_t launch_stress(const GridDev& g, const float* eps, float* sig, double* partials, int nblk,
                          cudaStream_t st) {
  const long long n4 = g.n / 4;
  k_stress<<<nblk, kRedThreads, 0, st>>>(reinterpret_cast<const float4*>(eps),
                                         reinterpret_cast<const uchar4*>(g.phase), g.cmat,
                                         reinterpret_cast<float4*>(sig), n4, partials, nblk);
  return cudaGetLastError();
}

// out = a x + b y (y nullable; out may alias x or y)
__global__ void __launch_bounds__(kRedThreads) k_axpby(float4* out, float a, const float4* x,
                                                       float b, const float4* y, long long total4) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total4;
       q += (long long)gridDim.x * blockDim.x) {
    const float4 u = x[q];
    float4 r = make_float4(a * u.x, a * u.y, a * u.z, a * u.w);
    if (y) {
      const float4 v = y[q];
      r = make_float4(fmaf(b, v.x, r.x), fmaf(b, v.y, r.y), fmaf(b, v.z, r.z), fmaf(b, v.w, r.w));
    }
    out[q] = r;
  }
}

cudaError_t launch_axpby(float* out, float a, const float* x, float b, const float* y, long long n,
                         cudaStream_t st) {
  const long long total4 = 6 * (n / 4);
  k_axpby<<<stream_blocks(total4), kRedThreads, 0, st>>>(
      reinterpret_cast<float4*>(out), a, reinterpret_cast<const float4*>(x), b,
      reinterpret_cast<const float4*>(y), total4);
  return cudaGetLastError();
}

// eps_next = (C + C0)^-1 : (s_a + C0 : eps_b), Algorithm 3, per voxel; the
// inverse of an isotropic stiffness (lam_s, mu_s) maps t to
// (t - k_s tr(t) I) h_s with k_s = lam_s / (3 lam_s + 2 mu_s), h_s = 1 / (2 mu_s),
// both precomputed per phase in the table (lam_a, mu_a, k_s, h_s).
__global__ void __launch_bounds__(kRedThreads) k_pol_post(const float4* __restrict__ eps,
                                                          const float4* __restrict__ epsb,
                                                          const uchar4* __restrict__ phase,
                                                          const float4* __restrict__ post,
                                                          float lam0, float mu0,
                                                          float4* __restrict__ out, long long n4) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const uchar4 ph = phase[q];
    const float4 pm[4] = {post[ph.x], post[ph.y], post[ph.z], post[ph.w]};
    float e[6][4], b[6][4];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float4 u = eps[c * n4 + q], v = epsb[c * n4 + q];
      e[c][0] = u.x; e[c][1] = u.y; e[c][2] = u.z; e[c][3] = u.w;
      b[c][0] = v.x; b[c][1] = v.y; b[c][2] = v.z; b[c][3] = v.w;
    }
    float o[6][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float tre = e[0][k] + e[1][k] + e[2][k];
      const float trb = b[0][k] + b[1][k] + b[2][k];
      float t[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) t[c] = 2.f * pm[k].y * e[c][k] + 2.f * mu0 * b[c][k];
#pragma unroll
      for (int c = 0; c < 3; ++c) t[c] += pm[k].x * tre + lam0 * trb;
      const float trt = t[0] + t[1] + t[2];
      const float sh = pm[k].z * trt, inv2mu = pm[k].w;
#pragma unroll
      for (int c = 0; c < 6; ++c) o[c][k] = (t[c] - (c < 3 ? sh : 0.f)) * inv2mu;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) out[c * n4 + q] = make_float4(o[c][0], o[c][1], o[c][2], o[c][3]);
  }
}

cudaError_t launch_polarization_post(const GridDev& g, const float4* post, const float* eps,
                                     const float* eps_b, float* out, cudaStream_t st) {
  const long long n4 = g.n / 4;
  k_pol_post<<<stream_blocks(n4), kRedThreads, 0, st>>>(
      reinterpret_cast<const float4*>(eps), reinterpret_cast<const float4*>(eps_b),
      reinterpret_cast<const uchar4*>(g.phase), post, g.lam0, g.mu0,
      reinterpret_cast<float4*>(out), n4);
  return cudaGetLastError();
}

__global__ void k_fill(float4* f, float e0, float e1, float e2, float e3, float e4, float e5,
                       long long n4) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 6 * n4;
       q += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(q / n4);
    const float v = c == 0 ? e0 : c == 1 ? e1 : c == 2 ? e2 : c == 3 ? e3 : c == 4 ? e4 : e5;
    f[q] = make_float4(v, v, v, v);
  }
}

cudaError_t launch_fill(float* f, const double E[6], long long n, cudaStream_t st) {
  const long long n4 = n / 4;
  k_fill<<<stream_blocks(6 * n4), kRedThreads, 0, st>>>(
      reinterpret_cast<float4*>(f), (float)E[0], (float)E[1], (float)E[2], (float)E[3],
      (float)E[4], (float)E[5], n4);
  return cudaGetLastError();
}

// Newton step on the unstable subspace (Eq. 3.11 with H = Z^T F_u Z):
// sums[0] = |xi - eps|^2, sums[1 + j] = zeta_j = <Z_j, xi>;  M = (I - H)^-1.
// z+ = z + M (zeta - z);  c = z+ - zeta (so eps_next = xi + Z c);  z_next = z+
// (z = Z^T eps of the current iterate; z_next = Z^T eps_next).
// res_out = sqrt(sums[0]) * inv_norm.
// Newton step of Eqs. 3.10-3.13 in reduced coordinates.  With
// d = zeta - z = Z^T (xi - eps) (sums[1..p], formed from the difference field)
// and M = (I - H)^-1, the new iterate eps+ = xi + Z (z+ - zeta) with
// z+ = z + M d needs only c = z+ - zeta = (M - I) d.
__global__ void k_newton(const double* __restrict__ sums, int p, const double* __restrict__ M,
                         double* __restrict__ c, double* res_out, double inv_norm) {
  __shared__ double d[kMaxBasis];
  for (int j = threadIdx.x; j < p; j += blockDim.x) d[j] = sums[1 + j];
  __syncthreads();
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    double s = -d[j];
    for (int k = 0; k < p; ++k) s += M[(size_t)j * p + k] * d[k];
    c[j] = s;
  }
  if (threadIdx.x == 0) res_out[0] = sqrt(sums[0]) * inv_norm;   // NaN stays NaN
}

cudaError_t launch_newton(const double* sums, int p, const double* M, double* c, double* res_out,
                          double inv_norm, cudaStream_t st) {
  if (p > kMaxBasis) return cudaErrorInvalidValue;
  k_newton<<<1, 256, 0, st>>>(sums, p, M, c, res_out, inv_norm);
  return cudaGetLastError();
}

}  // namespace rpm
