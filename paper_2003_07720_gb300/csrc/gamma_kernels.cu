// The Lippmann-Schwinger map of Section 2 as three fused passes over HBM.
//
//   pass A (one block per z-plane and tensor component):
//       tau = (C(x) - C0) : eps  (Eq. 2.3, isotropic phases), packed as
//       complex rows z_n = tau_2n + i tau_2n+1, forward FFT along x of
//       length nx/2, real-to-complex untangling, forward FFT along y;
//       writes the half spectrum in slot order.
//   pass B (one block per T consecutive (ky, kx) pencils, all 6 components):
//       forward FFT along z, eps_hat = -Gamma0_hat(xi) : tau_hat per
//       frequency (Eq. 2.5) with the zero frequency set to E n_vox, inverse
//       FFT along z.
//   pass C (one block per z-plane and component): inverse FFT along y,
//       complex-to-real tangling, inverse FFT along x of length nx/2, scale.
//
// Two generations of kernels implement the passes.  The fused ones
// (k_plane_fwd, k_pencil_green, k_plane_inv) serve the common sizes: their
// first and last register FFT steps read and write global memory directly
// (pass C takes its plane in one bulk asynchronous copy), the (un)tangling
// of the half-length x transform is fused into an x step, the real DC and
// Nyquist x columns travel as one complex column so that the y transforms
// run on exactly nx/2 columns, and in pass B the forward z step 2, the
// Green operator and the inverse z step 1 run in registers.  The original
// kernels (k_pass_a/b/c and the five-pass variant) serve the other sizes.
//
// The Green operator of the isotropic reference medium is evaluated on the
// fly from the unit wave vector n = xi/|xi|:
//   Gamma0_hat : tau_hat = sym(n (x) w),  w = (v - a n (n.v)) / mu0,
//   v = tau_hat n,  a = (lam0 + mu0) / (lam0 + 2 mu0),
// obtained from div(C0 : eps(u) + tau) = 0 in Fourier space.
#include "async_copy.cuh"
#include "fft_smem.cuh"
#include "rpm_internal.h"

namespace rpm {

constexpr int kThreads = 256;

template <int NX, int NY>
struct PlaneCfg {
  static constexpr int NXH = NX / 2;
  static constexpr int SX = NXH + 1;          // x slots of the half spectrum
  static constexpr int NYP = NY + 1;          // odd column stride in float2
  static constexpr int PLANE_F2 = SX * NYP;
  static constexpr int TAB_F2 = NXH + NY + SX;
};

// X_k from Z_k = a, Z_{M-k} = b (M = nx/2), w = W_nx^k:
// X_k = (a + conj b)/2 - (i/2) w (a - conj b)
__device__ __forceinline__ float2 r2c_post(float2 a, float2 b, float2 w) {
  const float2 s = make_float2(a.x + b.x, a.y - b.y);
  const float2 d = make_float2(a.x - b.x, a.y + b.y);
  const float2 u = cmul(w, d);
  return make_float2(0.5f * (s.x + u.y), 0.5f * (s.y - u.x));
}

// 2 Z_k from X_k = a, X_{M-k} = b, w = W_nx^k:
// 2 Z_k = (a + conj b) + i (a - conj b) conj(w)
__device__ __forceinline__ float2 c2r_pre(float2 a, float2 b, float2 w) {
  const float2 s = make_float2(a.x + b.x, a.y - b.y);
  const float2 d = make_float2(a.x - b.x, a.y + b.y);
  const float2 u = cmulc(d, w);
  return make_float2(s.x - u.y, s.y + u.x);
}

// Block size of the plane passes and the blocks per SM the register budget targets.
constexpr int kPlaneThreads = 256;
constexpr int kPlaneMinBlocks = 3;

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, kPlaneMinBlocks)
    k_pass_a(GridDev g, const float* __restrict__ in, float2* __restrict__ spec, int mode) {
  using C = PlaneCfg<NX, NY>;
  extern __shared__ float2 sm[];
  float2* P = sm;
  float2* twx = P + C::PLANE_F2;
  float2* twy = twx + C::NXH;
  float2* r2c = twy + NY;
  float2* dm = r2c + C::SX;
  const int c = blockIdx.x, z = blockIdx.y;
  for (int i = threadIdx.x; i < C::NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  for (int i = threadIdx.x; i < C::SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) dm[i] = g.dmat[i];   // any uint8 id is in range
  __syncthreads();

  const size_t n2 = (size_t)g.n / 2;                     // float2 per component
  const size_t z2 = (size_t)z * NY * C::NXH;             // plane offset in float2
  const float2* in2 = reinterpret_cast<const float2*>(in);
  const uchar2* ph2 = reinterpret_cast<const uchar2*>(g.phase) + z2;
  // Loads are issued in groups of U per thread before any use, so each thread
  // keeps several independent requests in flight (the plane is streamed once).
  constexpr int TOT = NY * C::NXH, U = 4;
  for (int base = threadIdx.x; base < TOT; base += U * kPlaneThreads) {
    float2 a[U], b[U], d[U];
    uchar2 ph[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kPlaneThreads;
      if (idx < TOT) {
        const size_t v = z2 + idx;
        if (mode == GM_RAW_TAU || c >= 3) {
          a[u] = in2[c * n2 + v];
        } else {
          a[u] = in2[v];
          b[u] = in2[n2 + v];
          d[u] = in2[2 * n2 + v];
        }
        if (mode != GM_RAW_TAU) ph[u] = ph2[idx];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kPlaneThreads;
      if (idx < TOT) {
        const int y = idx / C::NXH, h = idx - y * C::NXH;
        float2 t;
        if (mode == GM_RAW_TAU) {
          t = a[u];
        } else {
          const float2 d0 = dm[ph[u].x], d1 = dm[ph[u].y];
          if (c >= 3) {
            t = make_float2(2.f * d0.y * a[u].x, 2.f * d1.y * a[u].y);
          } else {
            const float2 e = c == 0 ? a[u] : (c == 1 ? b[u] : d[u]);
            t = make_float2(fmaf(d0.x, a[u].x + b[u].x + d[u].x, 2.f * d0.y * e.x),
                            fmaf(d1.x, a[u].y + b[u].y + d[u].y, 2.f * d1.y * e.y));
          }
        }
        P[h * C::NYP + y] = t;
      }
    }
  }
  __syncthreads();
  smem_fft<C::NXH, false, NY, 1, C::NYP>(P, twx);
  for (int t = threadIdx.x; t < NY * (C::NXH / 2 + 1); t += blockDim.x) {
    const int y = t % NY, k = t / NY;
    if (k == 0) {
      const float2 z0 = P[y];
      P[y] = make_float2(z0.x + z0.y, 0.f);
      P[C::NXH * C::NYP + y] = make_float2(z0.x - z0.y, 0.f);
    } else {
      const int kk = C::NXH - k;
      const int sk = slot_of<C::NXH>(k), skk = slot_of<C::NXH>(kk);
      const float2 a = P[sk * C::NYP + y], b = P[skk * C::NYP + y];
      P[sk * C::NYP + y] = r2c_post(a, b, r2c[k]);
      if (kk != k) P[skk * C::NYP + y] = r2c_post(b, a, r2c[kk]);
    }
  }
  __syncthreads();
  smem_fft<NY, false, C::SX, C::NYP, 1>(P, twy);
  float2* out = spec + ((size_t)c * g.nz + z) * g.plane;
  for (int idx = threadIdx.x; idx < NY * C::SX; idx += blockDim.x) {
    const int sy = idx / C::SX, sx = idx - sy * C::SX;
    out[idx] = P[sx * C::NYP + sy];
  }
}

template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, kPlaneMinBlocks)
    k_pass_c(GridDev g, const float2* __restrict__ spec, float* __restrict__ outp, float scale) {
  using C = PlaneCfg<NX, NY>;
  extern __shared__ float2 sm[];
  float2* P = sm;
  float2* twx = P + C::PLANE_F2;
  float2* twy = twx + C::NXH;
  float2* r2c = twy + NY;
  const int c = blockIdx.x, z = blockIdx.y;
  for (int i = threadIdx.x; i < C::NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  for (int i = threadIdx.x; i < C::SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  const float2* src = spec + ((size_t)c * g.nz + z) * g.plane;
  {
    constexpr int TOT = NY * C::SX, U = 8;
    for (int base = threadIdx.x; base < TOT; base += U * kPlaneThreads) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) v[u] = src[idx];
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * kPlaneThreads;
        if (idx < TOT) {
          const int sy = idx / C::SX, sx = idx - sy * C::SX;
          P[sx * C::NYP + sy] = v[u];
        }
      }
    }
  }
  __syncthreads();
  smem_fft<NY, true, C::SX, C::NYP, 1>(P, twy);
  for (int t = threadIdx.x; t < NY * (C::NXH / 2 + 1); t += blockDim.x) {
    const int y = t % NY, k = t / NY;
    if (k == 0) {
      P[y] = c2r_pre(P[y], P[C::NXH * C::NYP + y], make_float2(1.f, 0.f));
    } else {
      const int kk = C::NXH - k;
      const int sk = slot_of<C::NXH>(k), skk = slot_of<C::NXH>(kk);
      const float2 a = P[sk * C::NYP + y], b = P[skk * C::NYP + y];
      P[sk * C::NYP + y] = c2r_pre(a, b, r2c[k]);
      if (kk != k) P[skk * C::NYP + y] = c2r_pre(b, a, r2c[kk]);
    }
  }
  __syncthreads();
  smem_fft<C::NXH, true, NY, 1, C::NYP>(P, twx);
  const size_t n2 = (size_t)g.n / 2;
  float2* out2 = reinterpret_cast<float2*>(outp) + c * n2 + (size_t)z * NY * C::NXH;
  for (int idx = threadIdx.x; idx < NY * C::NXH; idx += blockDim.x) {
    const int y = idx / C::NXH, h = idx - y * C::NXH;
    out2[idx] = cscale(P[h * C::NYP + y], scale);
  }
}

struct GammaArgs {
  float En[6];       // E * n_vox (zero frequency of the strain in GM_FULL_MAP)
  float a;           // (lam0 + mu0) / (lam0 + 2 mu0)
  float inv_mu0;
};

// T consecutive (ky, kx) pencils per pass-B block: TT = 0 takes the default
// for the length (8 pencils = 64-byte rows at nz = 64 and 128; 16 at
// nz = 256, one 512-thread block per SM, measured 0.980 vs 1.012 ms per
// 256^3 apply with 8); the tile autotuner of rpm_create also tries half and
// twice the default (GridDev::pencil_t).
template <int NZ, int TT = 0>
struct PencilCfg {
  static constexpr int T = TT ? TT : (NZ >= 256 ? 16 : (NZ >= 64 ? 8 : 32));
  static constexpr int NZP = (NZ % 2 == 0) ? NZ + 1 : NZ;
};

// eps_hat = -Gamma0_hat(n) : tau_hat for one frequency (components 11 22 33 23 13 12)
__device__ __forceinline__ void green_apply(float2* t, float n1, float n2, float n3, float a,
                                            float inv_mu0) {
  float2 v1, v2, v3;
  v1.x = t[0].x * n1 + t[5].x * n2 + t[4].x * n3;
  v1.y = t[0].y * n1 + t[5].y * n2 + t[4].y * n3;
  v2.x = t[5].x * n1 + t[1].x * n2 + t[3].x * n3;
  v2.y = t[5].y * n1 + t[1].y * n2 + t[3].y * n3;
  v3.x = t[4].x * n1 + t[3].x * n2 + t[2].x * n3;
  v3.y = t[4].y * n1 + t[3].y * n2 + t[2].y * n3;
  const float sx = n1 * v1.x + n2 * v2.x + n3 * v3.x;
  const float sy = n1 * v1.y + n2 * v2.y + n3 * v3.y;
  float2 w1, w2, w3;
  w1.x = (v1.x - a * n1 * sx) * inv_mu0;
  w1.y = (v1.y - a * n1 * sy) * inv_mu0;
  w2.x = (v2.x - a * n2 * sx) * inv_mu0;
  w2.y = (v2.y - a * n2 * sy) * inv_mu0;
  w3.x = (v3.x - a * n3 * sx) * inv_mu0;
  w3.y = (v3.y - a * n3 * sy) * inv_mu0;
  t[0] = make_float2(-n1 * w1.x, -n1 * w1.y);
  t[1] = make_float2(-n2 * w2.x, -n2 * w2.y);
  t[2] = make_float2(-n3 * w3.x, -n3 * w3.y);
  t[3] = make_float2(-0.5f * (n2 * w3.x + n3 * w2.x), -0.5f * (n2 * w3.y + n3 * w2.y));
  t[4] = make_float2(-0.5f * (n1 * w3.x + n3 * w1.x), -0.5f * (n1 * w3.y + n3 * w1.y));
  t[5] = make_float2(-0.5f * (n1 * w2.x + n2 * w1.x), -0.5f * (n1 * w2.y + n2 * w1.y));
}

// Pass B body for NT threads per block (k_pass_b: 256; k_pass_b_wide: 512,
// where shared memory limits a block of 256 to two blocks per SM, nz >= 256,
// so that 32 warps per SM hide the latency).
template <int NZ, int TT, int NT>
__device__ __forceinline__ void pass_b_body(const GridDev& g, float2* __restrict__ spec, int mode,
                                            const GammaArgs& ga) {
  using C = PencilCfg<NZ, TT>;
  constexpr int T = C::T, NZP = C::NZP;
  constexpr int Z1 = Split<NZ>::N1, Z2 = Split<NZ>::N2;
  // two register steps: the first reads the spectrum and the last writes it
  // straight from / to global memory (task q -> pencil t fastest, then
  // component, then n2, so a half-warp covers two components' lines)
  constexpr bool DIRECT = Z2 > 1;
  extern __shared__ float2 sm[];
  float2* B = sm;
  float2* twz = B + 6 * T * NZP;
  __shared__ float4 pen[T];          // per pencil: (xi_x, xi_y, has-Nyquist, non-zero count)
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) twz[i] = g.tw_z[i];
  const int m0 = blockIdx.x * T;
  const int plane = g.plane;
  if (threadIdx.x < T) {
    const int m = m0 + threadIdx.x;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < plane) {
      const int sxn = g.nxh + 1;
      const int sy = m / sxn, sx = m - sy * sxn;
      const int2 fx = g.fx[sx], fy = g.fy[sy];
      q = make_float4(fx.x * g.inv_lx, fy.x * g.inv_ly, (float)(fx.y | fy.y),
                      (float)((fx.x != 0) + (fy.x != 0)));
    }
    pen[threadIdx.x] = q;
  }
  if constexpr (DIRECT) {
    __syncthreads();
    for (int q = threadIdx.x; q < 6 * T * Z2; q += NT) {
      const int t = q % T, c = (q / T) % 6, n2 = q / (6 * T);
      const int m = m0 + t;
      const float2* src = spec + ((size_t)c * NZ + n2) * plane + m;
      const size_t zs = (size_t)Z2 * plane;
      float2 v[Z1];
#pragma unroll
      for (int i = 0; i < Z1; ++i) v[i] = m < plane ? src[i * zs] : make_float2(0.f, 0.f);
      RegDft<Z1, false>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < Z1; ++k1) v[k1] = cmul(v[k1], twz[n2 * Z1 + k1]);
      float2* p = B + (c * T + t) * NZP + n2;
#pragma unroll
      for (int i = 0; i < Z1; ++i) p[i * Z2] = v[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 6 * T * Z1; q += NT) {   // forward step 2 in shared memory
      const int b = q % (6 * T), k1 = q / (6 * T);
      float2* p = B + b * NZP + k1 * Z2;
      float2 v[Z2];
#pragma unroll
      for (int i = 0; i < Z2; ++i) v[i] = p[i];
      RegDft<Z2, false>::run(v);
#pragma unroll
      for (int i = 0; i < Z2; ++i) p[i] = v[i];
    }
    __syncthreads();
  } else {
    constexpr int TOT = 6 * NZ * T, U = 8;
    for (int base = threadIdx.x; base < TOT; base += U * NT) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NT;
        const int t = idx % T, r = idx / T, z = r % NZ, c = r / NZ;
        const int m = m0 + t;
        v[u] = (idx < TOT && m < plane) ? spec[((size_t)c * NZ + z) * plane + m]
                                        : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NT;
        if (idx < TOT) {
          const int t = idx % T, r = idx / T, z = r % NZ, c = r / NZ;
          B[(c * T + t) * NZP + z] = v[u];
        }
      }
    }
    __syncthreads();
    smem_fft<NZ, false, 6 * T, NZP, 1>(B, twz);
  }
  for (int idx = threadIdx.x; idx < T * NZ; idx += blockDim.x) {
    const int sz = idx % NZ, t = idx / NZ;
    if (m0 + t >= plane) continue;
    const float4 q = pen[t];
    const int kz = freq_of<NZ>(sz);
    const int mz = (2 * kz < NZ) ? kz : kz - NZ;
    const bool nyqz = (NZ % 2 == 0) && NZ > 1 && (2 * kz == NZ);
    float2 tv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) tv[c] = B[(c * T + t) * NZP + sz];
    const int nnz = (int)q.w + (mz != 0);
    if (nnz == 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c)
        tv[c] = make_float2(mode == GM_FULL_MAP ? ga.En[c] : 0.f, 0.f);
    } else if (g.nyquist == 0 && nnz >= 2 && (q.z != 0.f || nyqz)) {
#pragma unroll
      for (int c = 0; c < 6; ++c) tv[c] = make_float2(0.f, 0.f);
    } else {
      const float x1 = q.x, x2 = q.y, x3 = mz * g.inv_lz;
      const float inv = rsqrtf(x1 * x1 + x2 * x2 + x3 * x3);
      green_apply(tv, x1 * inv, x2 * inv, x3 * inv, ga.a, ga.inv_mu0);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) B[(c * T + t) * NZP + sz] = tv[c];
  }
  __syncthreads();
  if constexpr (DIRECT) {
    for (int q = threadIdx.x; q < 6 * T * Z1; q += NT) {   // inverse step 1 in shared memory
      const int b = q % (6 * T), k1 = q / (6 * T);
      float2* p = B + b * NZP + k1 * Z2;
      float2 v[Z2];
#pragma unroll
      for (int i = 0; i < Z2; ++i) v[i] = p[i];
      RegDft<Z2, true>::run(v);
#pragma unroll
      for (int n2 = 1; n2 < Z2; ++n2) v[n2] = cmulc(v[n2], twz[n2 * Z1 + k1]);
#pragma unroll
      for (int i = 0; i < Z2; ++i) p[i] = v[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 6 * T * Z2; q += NT) {   // inverse step 2 -> global
      const int t = q % T, c = (q / T) % 6, n2 = q / (6 * T);
      const int m = m0 + t;
      const float2* p = B + (c * T + t) * NZP + n2;
      float2 v[Z1];
#pragma unroll
      for (int i = 0; i < Z1; ++i) v[i] = p[i * Z2];
      RegDft<Z1, true>::run(v);
      if (m < plane) {
        float2* dst = spec + ((size_t)c * NZ + n2) * plane + m;
        const size_t zs = (size_t)Z2 * plane;
#pragma unroll
        for (int i = 0; i < Z1; ++i) dst[i * zs] = v[i];
      }
    }
  } else {
    smem_fft<NZ, true, 6 * T, NZP, 1>(B, twz);
    for (int idx = threadIdx.x; idx < 6 * NZ * T; idx += blockDim.x) {
      const int t = idx % T, r = idx / T, z = r % NZ, c = r / NZ;
      const int m = m0 + t;
      if (m < plane) spec[((size_t)c * NZ + z) * plane + m] = B[(c * T + t) * NZP + z];
    }
  }
}

template <int NZ, int TT>
__global__ void __launch_bounds__(kThreads) k_pass_b(GridDev g, float2* __restrict__ spec, int mode,
                                                     GammaArgs ga) {
  pass_b_body<NZ, TT, kThreads>(g, spec, mode, ga);
}

template <int NZ, int TT>
__global__ void __launch_bounds__(2 * kThreads, 2) k_pass_b_wide(GridDev g,
                                                                float2* __restrict__ spec,
                                                                int mode, GammaArgs ga) {
  pass_b_body<NZ, TT, 2 * kThreads>(g, spec, mode, ga);
}


// ---------------------------------------------------------------------------
// Fused-step kernels (square planes nx = ny in {48, 64, 96, 128}; pencils of
// length nz with 128 / split_n1(nz) pencils per block, nz in {32, 48, 96, 128}).
// ---------------------------------------------------------------------------

// Row task q of an x step over NY rows: (y, n2).  With N2 = 8 the two
// half-warps take rows y and y + 8, so that the 8-byte accesses of one
// instruction fall in distinct banks (row stride nx/2 + 1 float2).
template <int N2, int NY>
__device__ __forceinline__ void row_task(int q, int& y, int& n2) {
  if (N2 == 8 && NY % 16 == 0) {
    n2 = q & 7;
    const int h = (q >> 3) & 1, g = q >> 4;
    y = (g & 7) + ((g >> 3) << 4) + (h << 3);
  } else {
    n2 = q % N2;
    y = q / N2;
  }
}

// Pass A, one block per (z, component).  x step 1 reads the strain rows from
// global memory and forms tau on the way in; x step 2 is fused with the
// real-to-complex untangling; the (real) DC and Nyquist x columns are stored
// together as X_0 + i X_nx/2 in column 0, so the y transform runs on nx/2
// columns; y step 2 writes the spectrum plane to global memory, and the
// packed column is separated last (A_k = (C_k + conj C_-k) / 2,
// B_k = (C_k - conj C_-k) / 2i).
// 16-point x steps (nx = 96) need more registers than three blocks per SM allow
template <int NX, int NY>
__global__ void __launch_bounds__(kPlaneThreads, Split<NX / 2>::N1 >= 16 ? 2 : kPlaneMinBlocks)
    k_plane_fwd(GridDev g, const float* __restrict__ in, float2* __restrict__ spec, int mode) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  constexpr int X1 = Split<NXH>::N1, X2 = Split<NXH>::N2;
  constexpr int Y1 = Split<NY>::N1, Y2 = Split<NY>::N2;
  static_assert(X2 > 1 && X1 % 2 == 0, "x split must have two steps and an even first factor");
  extern __shared__ __align__(128) float2 sm[];
  float2* P = sm;                      // [NY][SX]: the spectrum plane's own layout
  float2* twx = P + NY * SX;           // transposed: W^(n2 k1) at k1 * X2 + n2
  float2* twy = twx + NXH;
  float2* r2c = twy + NY;
  float2* dm = r2c + SX;
  const int c = blockIdx.x, z = blockIdx.y;
  allow_dependent_launch();
  for (int i = threadIdx.x; i < NXH; i += blockDim.x)
    twx[(i % X1) * X2 + i / X1] = g.tw_x[i];
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  for (int i = threadIdx.x; i < SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  grid_dependency_wait();   // the FFT tables are fixed; everything below may be in flight
  for (int i = threadIdx.x; i < 256; i += blockDim.x) dm[i] = g.dmat[i];
  __syncthreads();
  const size_t nf2 = (size_t)g.n / 2;
  const float2* in2 = reinterpret_cast<const float2*>(in) + (size_t)z * NY * NXH;
  const uchar2* ph2 = reinterpret_cast<const uchar2*>(g.phase) + (size_t)z * NY * NXH;
  const bool three = mode != GM_RAW_TAU && c < 3;
  // With at most two phases the material table is two register pairs and a
  // select (phase ids are < n_phases), which takes the table lookups off the
  // shared-memory pipe.
  const bool two = g.n_phases <= 2;
  const float2 dm0 = dm[0], dm1 = dm[1];
  auto dmat = [&](unsigned char id) { return two ? (id ? dm1 : dm0) : dm[id]; };
  for (int q = threadIdx.x; q < NY * X2; q += blockDim.x) {
    int y, n2;
    row_task<X2, NY>(q, y, n2);
    const int rb = y * NXH + n2;
    float2 v[X1];
    if (!three) {
      float2 a[X1];
      uchar2 ph[X1];
#pragma unroll
      for (int i = 0; i < X1; ++i) {
        a[i] = in2[c * nf2 + rb + X2 * i];
        if (mode != GM_RAW_TAU) ph[i] = ph2[rb + X2 * i];
      }
#pragma unroll
      for (int i = 0; i < X1; ++i) {
        if (mode == GM_RAW_TAU) {
          v[i] = a[i];
        } else {
          const float2 d0 = dmat(ph[i].x), d1 = dmat(ph[i].y);
          v[i] = make_float2(2.f * d0.y * a[i].x, 2.f * d1.y * a[i].y);
        }
      }
    } else {
      constexpr int H = X1 >= 4 ? 4 : X1;   // voxel pairs loaded per batch
#pragma unroll
      for (int i0 = 0; i0 < X1; i0 += H) {
        float2 a[H], b[H], d[H];
        uchar2 ph[H];
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const int i = i0 + j;
          a[j] = in2[rb + X2 * i];
          b[j] = in2[nf2 + rb + X2 * i];
          d[j] = in2[2 * nf2 + rb + X2 * i];
          ph[j] = ph2[rb + X2 * i];
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
          const float2 d0 = dmat(ph[j].x), d1 = dmat(ph[j].y);
          const float2 e = c == 0 ? a[j] : (c == 1 ? b[j] : d[j]);
          v[i0 + j] = make_float2(fmaf(d0.x, a[j].x + b[j].x + d[j].x, 2.f * d0.y * e.x),
                                  fmaf(d1.x, a[j].y + b[j].y + d[j].y, 2.f * d1.y * e.y));
        }
      }
    }
    RegDft<X1, false>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < X1; ++k1) v[k1] = cmul(v[k1], twx[k1 * X2 + n2]);
    float2* p = P + y * SX + n2;
#pragma unroll
    for (int i = 0; i < X1; ++i) p[i * X2] = v[i];
  }
  __syncthreads();
  // x step 2 fused with the untangling.  Slot group k1 holds the
  // frequencies k1 + X1 i; the partner nx/2 - k of k lies in group X1 - k1
  // (groups 0 and X1/2 pair with themselves).
  constexpr int NU = X1 / 2 + 1;
  for (int t = threadIdx.x; t < NY * NU; t += blockDim.x) {
    const int b = t % NY, u = t / NY;
    float2* p = P + b * SX;
    if (u == 0 || u == X1 / 2) {
      const int k1 = u;
      float2 v[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) v[i] = p[k1 * X2 + i];
      RegDft<X2, false>::run(v);
      float2 o[X2];
      if (k1 == 0) {
        const float2 z0 = v[0];
        o[0] = make_float2(z0.x + z0.y, z0.x - z0.y);   // (X_0, X_nx/2), both real
#pragma unroll
        for (int i = 1; i < X2; ++i) {
          const int ip = X2 - i;
          if (i < ip) {
            o[i] = r2c_post(v[i], v[ip], r2c[X1 * i]);
            o[ip] = r2c_post(v[ip], v[i], r2c[X1 * ip]);
          } else if (i == ip) {
            o[i] = r2c_post(v[i], v[i], r2c[X1 * i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < X2; ++i) {
          const int ip = X2 - 1 - i;
          if (i < ip) {
            o[i] = r2c_post(v[i], v[ip], r2c[X1 / 2 + X1 * i]);
            o[ip] = r2c_post(v[ip], v[i], r2c[X1 / 2 + X1 * ip]);
          } else if (i == ip) {
            o[i] = r2c_post(v[i], v[i], r2c[X1 / 2 + X1 * i]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < X2; ++i) p[k1 * X2 + i] = o[i];
    } else {
      const int k1 = u, k1p = X1 - u;
      float2 va[X2], vb[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        va[i] = p[k1 * X2 + i];
        vb[i] = p[k1p * X2 + i];
      }
      RegDft<X2, false>::run(va);
      RegDft<X2, false>::run(vb);
      float2 oa[X2], ob[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        const int ip = X2 - 1 - i;
        oa[i] = r2c_post(va[i], vb[ip], r2c[k1 + X1 * i]);
        ob[ip] = r2c_post(vb[ip], va[i], r2c[k1p + X1 * ip]);
      }
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        p[k1 * X2 + i] = oa[i];
        p[k1p * X2 + i] = ob[i];
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NXH * Y2; t += blockDim.x) {   // y step 1
    const int b = t % NXH, n2 = t / NXH;
    float2* p = P + b + n2 * SX;
    float2 v[Y1];
#pragma unroll
    for (int i = 0; i < Y1; ++i) v[i] = p[i * Y2 * SX];
    RegDft<Y1, false>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < Y1; ++k1) v[k1] = cmul(v[k1], twy[n2 * Y1 + k1]);
#pragma unroll
    for (int i = 0; i < Y1; ++i) p[i * Y2 * SX] = v[i];
  }
  __syncthreads();
  float2* out = spec + ((size_t)c * g.nz + z) * g.plane;
  for (int t = threadIdx.x; t < NXH * Y1; t += blockDim.x) {   // y step 2 -> global
    const int b = t % NXH, k1 = t / NXH;
    float2* p = P + b + k1 * Y2 * SX;
    float2 v[Y2];
#pragma unroll
    for (int i = 0; i < Y2; ++i) v[i] = p[i * SX];
    RegDft<Y2, false>::run(v);
    if (b == 0) {
#pragma unroll
      for (int i = 0; i < Y2; ++i) p[i * SX] = v[i];
    } else {
#pragma unroll
      for (int i = 0; i < Y2; ++i) out[(size_t)(k1 * Y2 + i) * SX + b] = v[i];
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < NY; s += blockDim.x) {   // separate the packed column
    const int k = freq_of<NY>(s);
    const int sn = slot_of<NY>((NY - k) % NY);
    const float2 a = P[s * SX], b = P[sn * SX];
    out[(size_t)s * SX] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    out[(size_t)s * SX + NXH] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
  }
}

// Algorithm 3's last step at one voxel: out = (C + C0)^-1 : (s_a + C0 : eps_b)
// with s_a = lam_a tr(eps) I + 2 mu_a eps and (C + C0) = (lam_s, mu_s); the
// inverse of an isotropic stiffness maps t to (t - k_s tr(t) I) h_s with
// k_s = lam_s / (3 lam_s + 2 mu_s), h_s = 1 / (2 mu_s).  pm = (lam_a, mu_a,
// k_s, h_s) of the voxel's phase.
__device__ __forceinline__ void post_normal(const float e[3], const float b[3], float4 pm,
                                            float lam0, float mu0, float o[3]) {
  const float tre = e[0] + e[1] + e[2];
  const float trb = b[0] + b[1] + b[2];
  float t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    t[k] = 2.f * pm.y * e[k] + 2.f * mu0 * b[k];
    t[k] += pm.x * tre + lam0 * trb;
  }
  const float sh = pm.z * (t[0] + t[1] + t[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) o[k] = (t[k] - sh) * pm.w;
}

__device__ __forceinline__ float post_shear(float e, float b, float4 pm, float mu0) {
  return (2.f * pm.y * e + 2.f * mu0 * b) * pm.w;
}

// Pass C, one block per (component, z).  The spectrum plane arrives by one
// bulk asynchronous copy; y step 1 packs the DC and Nyquist x columns as
// X_0 + i X_nx/2 (their inverse y transforms are real, so the result holds
// both in its real and imaginary parts); the tangling is fused into x step
// 1; x step 2 writes the real rows to global memory, scaled.  Without POST
// a non-null `eps` is a field added to the output on the way out (the
// defect of a re-centred iterate).
//
// POST: the pass ends with Algorithm 3's post-step instead (Section 5.5),
// the transformed planes being eps_b and `eps` the map's input.  Blocks are
// numbered z * 6 + c and run in clusters of three: the shear blocks apply
// the post-step to their own component on the way out; the three normal
// blocks of a plane, which need tr(eps_b), keep their real planes in shared
// memory and each finishes all three normal components on a third of the
// plane, reading the other two planes from the cluster's shared memory.
template <int NX, int NY, bool POST>
__global__ void __launch_bounds__(kPlaneThreads, kPlaneMinBlocks)
    k_plane_inv(GridDev g, const float2* __restrict__ spec, float* __restrict__ outp,
                float scale, const float* __restrict__ eps, const float4* __restrict__ post) {
  constexpr int NXH = NX / 2, SX = NXH + 1, PL = NY * SX;
  constexpr int X1 = Split<NXH>::N1, X2 = Split<NXH>::N2;
  constexpr int Y1 = Split<NY>::N1, Y2 = Split<NY>::N2;
  static_assert(X2 > 1 && X1 % 2 == 0, "x split must have two steps and an even first factor");
  static_assert((PL * 8) % 16 == 0, "bulk copy size");
  extern __shared__ __align__(128) float2 sm[];
  float2* P = sm;
  float2* twx = P + PL;
  float2* twy = twx + NXH;
  float2* r2c = twy + NY;
  float4* pt = reinterpret_cast<float4*>(r2c + SX + ((PL + NXH + NY + SX) & 1));   // POST
  __shared__ __align__(8) uint64_t bar;
  __shared__ int fail;
  const int c = POST ? (int)blockIdx.x % 6 : (int)blockIdx.x / g.nz;
  const int z = POST ? (int)blockIdx.x / 6 : (int)blockIdx.x - c * g.nz;
  const int item = c * g.nz + z;
  const bool gather = POST && c < 3;   // a normal block of a post-step cluster
  allow_dependent_launch();
  if (threadIdx.x == 0) {
    fail = 0;
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  for (int i = threadIdx.x; i < NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  for (int i = threadIdx.x; i < SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  if (POST)
    for (int i = threadIdx.x; i < 256; i += blockDim.x) pt[i] = post[i];
  grid_dependency_wait();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, PL * 8);
    bulk_load(P, spec + (size_t)item * g.plane, PL * 8, &bar);
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0)) fail = 1;
  __syncthreads();
  if (fail) {   // the copy never completed: record it and leave the plane alone
    if (threadIdx.x == 0) {
      atomicExch(g.err, 1);
      mbar_wait(&bar, 0);
    }
    if (gather) {   // the cluster's two barriers are still met
      cluster_sync();
      cluster_sync();
    }
    return;
  }
  for (int t = threadIdx.x; t < NXH * Y1; t += blockDim.x) {   // y step 1 (inverse)
    const int b = t % NXH, k1 = t / NXH;
    float2* p = P + k1 * Y2 * SX + b;
    float2 v[Y2];
#pragma unroll
    for (int i = 0; i < Y2; ++i) v[i] = p[i * SX];
    if (b == 0) {
#pragma unroll
      for (int i = 0; i < Y2; ++i) {
        const float2 w = p[i * SX + NXH];
        v[i] = make_float2(v[i].x - w.y, v[i].y + w.x);
      }
    }
    RegDft<Y2, true>::run(v);
#pragma unroll
    for (int n2 = 1; n2 < Y2; ++n2) v[n2] = cmulc(v[n2], twy[n2 * Y1 + k1]);
#pragma unroll
    for (int i = 0; i < Y2; ++i) p[i * SX] = v[i];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NXH * Y2; t += blockDim.x) {   // y step 2 (inverse)
    const int b = t % NXH, n2 = t / NXH;
    float2* p = P + b + n2 * SX;
    float2 v[Y1];
#pragma unroll
    for (int i = 0; i < Y1; ++i) v[i] = p[i * Y2 * SX];
    RegDft<Y1, true>::run(v);
#pragma unroll
    for (int i = 0; i < Y1; ++i) p[i * Y2 * SX] = v[i];
  }
  __syncthreads();
  constexpr int NU = X1 / 2 + 1;   // tangling fused into x step 1 (inverse)
  for (int t = threadIdx.x; t < NY * NU; t += blockDim.x) {
    const int b = t % NY, u = t / NY;
    float2* p = P + b * SX;
    if (u == 0 || u == X1 / 2) {
      const int k1 = u;
      float2 v[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) v[i] = p[k1 * X2 + i];
      float2 o[X2];
      if (k1 == 0) {
        o[0] = make_float2(v[0].x + v[0].y, v[0].x - v[0].y);   // from (x_DC, x_Nyquist)
#pragma unroll
        for (int i = 1; i < X2; ++i) {
          const int ip = X2 - i;
          if (i < ip) {
            o[i] = c2r_pre(v[i], v[ip], r2c[X1 * i]);
            o[ip] = c2r_pre(v[ip], v[i], r2c[X1 * ip]);
          } else if (i == ip) {
            o[i] = c2r_pre(v[i], v[i], r2c[X1 * i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < X2; ++i) {
          const int ip = X2 - 1 - i;
          if (i < ip) {
            o[i] = c2r_pre(v[i], v[ip], r2c[X1 / 2 + X1 * i]);
            o[ip] = c2r_pre(v[ip], v[i], r2c[X1 / 2 + X1 * ip]);
          } else if (i == ip) {
            o[i] = c2r_pre(v[i], v[i], r2c[X1 / 2 + X1 * i]);
          }
        }
      }
      RegDft<X2, true>::run(o);
#pragma unroll
      for (int n2 = 1; n2 < X2; ++n2) o[n2] = cmulc(o[n2], twx[n2 * X1 + k1]);
#pragma unroll
      for (int i = 0; i < X2; ++i) p[k1 * X2 + i] = o[i];
    } else {
      const int k1 = u, k1p = X1 - u;
      float2 va[X2], vb[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        va[i] = p[k1 * X2 + i];
        vb[i] = p[k1p * X2 + i];
      }
      float2 oa[X2], ob[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        const int ip = X2 - 1 - i;
        oa[i] = c2r_pre(va[i], vb[ip], r2c[k1 + X1 * i]);
        ob[ip] = c2r_pre(vb[ip], va[i], r2c[k1p + X1 * ip]);
      }
      RegDft<X2, true>::run(oa);
      RegDft<X2, true>::run(ob);
#pragma unroll
      for (int n2 = 1; n2 < X2; ++n2) {
        oa[n2] = cmulc(oa[n2], twx[n2 * X1 + k1]);
        ob[n2] = cmulc(ob[n2], twx[n2 * X1 + k1p]);
      }
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        p[k1 * X2 + i] = oa[i];
        p[k1p * X2 + i] = ob[i];
      }
    }
  }
  __syncthreads();
  const size_t nf2 = (size_t)g.n / 2, zoff = (size_t)z * NY * NXH;
  float2* out2 = reinterpret_cast<float2*>(outp) + zoff;
  const float2* e2 = reinterpret_cast<const float2*>(eps) + zoff;
  const uchar2* ph2 = reinterpret_cast<const uchar2*>(g.phase) + zoff;
  for (int q = threadIdx.x; q < NY * X2; q += blockDim.x) {   // x step 2 (inverse)
    int y, n2;
    row_task<X2, NY>(q, y, n2);
    float2* p = P + y * SX + n2;
    const int r = y * NXH + n2;
    float2 ev[X1];   // shear post-step: the map's input and phases, loaded ahead
    uchar2 pv[X1];   // of the transform where the registers allow
    constexpr bool AHEAD = X1 <= 8;
    const bool addend = !POST && eps != nullptr;
    if ((POST || addend) && AHEAD && !gather) {
#pragma unroll
      for (int i = 0; i < X1; ++i) {
        ev[i] = e2[c * nf2 + r + i * X2];
        if (POST) pv[i] = ph2[r + i * X2];
      }
    }
    float2 v[X1];
#pragma unroll
    for (int i = 0; i < X1; ++i) v[i] = p[i * X2];
    RegDft<X1, true>::run(v);
    if (!POST && addend) {   // -> global, with the added field
#pragma unroll
      for (int i = 0; i < X1; ++i) {
        if (!AHEAD) ev[i] = e2[c * nf2 + r + i * X2];
        const float2 b = cscale(v[i], scale);
        out2[c * nf2 + r + i * X2] = make_float2(b.x + ev[i].x, b.y + ev[i].y);
      }
    } else if (!POST) {   // -> global
#pragma unroll
      for (int i = 0; i < X1; ++i) out2[c * nf2 + r + i * X2] = cscale(v[i], scale);
    } else if (gather) {   // -> the block's own slots, for the cluster's post-step
#pragma unroll
      for (int i = 0; i < X1; ++i) p[i * X2] = cscale(v[i], scale);
    } else {   // shear component: post-step on the way out
#pragma unroll
      for (int i = 0; i < X1; ++i) {
        if (!AHEAD) {
          ev[i] = e2[c * nf2 + r + i * X2];
          pv[i] = ph2[r + i * X2];
        }
        const float2 b = cscale(v[i], scale);
        out2[c * nf2 + r + i * X2] = make_float2(post_shear(ev[i].x, b.x, pt[pv[i].x], g.mu0),
                                                 post_shear(ev[i].y, b.y, pt[pv[i].y], g.mu0));
      }
    }
  }
  if (!gather) return;
  // eps_b of the three normal components sits in the cluster's blocks 0, 1, 2
  // (rank = c), at slot y * SX + h for the float2 pair h of row y.  Each
  // thread takes U float2 pairs at a time, all loads issued before any use.
  cluster_sync();
  uint32_t rb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) rb[k] = cluster_map(P, (uint32_t)k);
  constexpr int U = 4, STRIDE = 3 * kPlaneThreads, TOT = NY * NXH;
  for (int f0 = threadIdx.x + c * kPlaneThreads; f0 < TOT; f0 += U * STRIDE) {
    float2 b[U][3], e[U][3];
    uchar2 ph[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + u * STRIDE;
      if (f < TOT) {
        const int s = f + f / NXH;   // y * SX + h
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          b[u][k] = ld_cluster_f2(rb[k] + 8u * (uint32_t)s);
          e[u][k] = e2[k * nf2 + f];
        }
        ph[u] = ph2[f];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int f = f0 + u * STRIDE;
      if (f < TOT) {
        const float ex[3] = {e[u][0].x, e[u][1].x, e[u][2].x};
        const float ey[3] = {e[u][0].y, e[u][1].y, e[u][2].y};
        const float bx[3] = {b[u][0].x, b[u][1].x, b[u][2].x};
        const float by[3] = {b[u][0].y, b[u][1].y, b[u][2].y};
        float ox[3], oy[3];
        post_normal(ex, bx, pt[ph[u].x], g.lam0, g.mu0, ox);
        post_normal(ey, by, pt[ph[u].y], g.lam0, g.mu0, oy);
#pragma unroll
        for (int k = 0; k < 3; ++k) out2[k * nf2 + f] = make_float2(ox[k], oy[k]);
      }
    }
  }
  cluster_sync();   // no block leaves while another still reads its planes
}

// Pass B with T = 128 / split_n1(nz) pencils per block and 256 threads.
// Forward z step 1 reads the spectrum from global memory; forward step 2, the
// Green operator and inverse step 1 run in registers on one (pencil, k1)
// group per pair of threads, lanes l and l + 16 holding the normal and the
// shear components of the same frequencies and exchanging their partial sums
// of tau_hat n with one shuffle per value; inverse step 2 writes back to
// global memory.
template <int NZ>
struct PencilFused {
  static constexpr int Z1 = Split<NZ>::N1, Z2 = Split<NZ>::N2;
  static constexpr int T = 128 / Z1;
  static constexpr int NZP = NZ + 1;
};

template <int NZ>
__global__ void __launch_bounds__(kThreads, 3) k_pencil_green(GridDev g, float2* __restrict__ spec,
                                                             int mode, GammaArgs ga) {
  using C = PencilFused<NZ>;
  constexpr int Z1 = C::Z1, Z2 = C::Z2, T = C::T, NZP = C::NZP;
  static_assert(T * Z1 * 2 == kThreads, "one thread pair per (pencil, k1) group");
  extern __shared__ __align__(128) float2 sm[];
  float2* B = sm;                       // [6][T][NZP]
  float2* twz = B + 6 * T * NZP;
  __shared__ float4 pen[T];             // per pencil: (xi_x, xi_y, has-Nyquist, non-zero count)
  const int m0 = blockIdx.x * T;
  const int plane = g.plane;
  allow_dependent_launch();
  for (int i = threadIdx.x; i < NZ; i += blockDim.x) twz[i] = g.tw_z[i];
  if (threadIdx.x < T) {
    const int m = m0 + threadIdx.x;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < plane) {
      const int sxn = g.nxh + 1;
      const int sy = m / sxn, sx = m - sy * sxn;
      const int2 fx = g.fx[sx], fy = g.fy[sy];
      q = make_float4(fx.x * g.inv_lx, fy.x * g.inv_ly, (float)(fx.y | fy.y),
                      (float)((fx.x != 0) + (fy.x != 0)));
    }
    pen[threadIdx.x] = q;
  }
  grid_dependency_wait();
  __syncthreads();
  // forward step 1; task q -> (pencil t fastest, then component, then n2):
  // a half-warp covers two components, whose lines are 16 words apart in banks
  for (int q = threadIdx.x; q < 6 * T * Z2; q += blockDim.x) {
    const int t = q % T, c = (q / T) % 6, n2 = q / (6 * T);
    const int m = m0 + t;
    const float2* src = spec + ((size_t)c * NZ + n2) * plane + m;
    const size_t zs = (size_t)Z2 * plane;
    float2 v[Z1];
#pragma unroll
    for (int i = 0; i < Z1; ++i) v[i] = m < plane ? src[i * zs] : make_float2(0.f, 0.f);
    RegDft<Z1, false>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < Z1; ++k1) v[k1] = cmul(v[k1], twz[n2 * Z1 + k1]);
    float2* p = B + (c * T + t) * NZP + n2;
#pragma unroll
    for (int i = 0; i < Z1; ++i) p[i * Z2] = v[i];
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int pi = w * 16 + (lane & 15);
    const int h = lane >> 4;             // 0: tau11 tau22 tau33, 1: tau23 tau13 tau12
    const int t = pi % T, k1 = pi / T;
    float2 v[3][Z2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2* p = B + ((3 * h + j) * T + t) * NZP + k1 * Z2;
#pragma unroll
      for (int i = 0; i < Z2; ++i) v[j][i] = p[i];
      RegDft<Z2, false>::run(v[j]);
    }
    const float4 q = pen[t];
#pragma unroll
    for (int k2 = 0; k2 < Z2; ++k2) {
      const int kz = k1 + Z1 * k2;
      const int mz = (2 * kz < NZ) ? kz : kz - NZ;
      const bool nyqz = (NZ % 2 == 0) && (2 * kz == NZ);
      const int nnz = (int)q.w + (mz != 0);
      const bool zero_f = nnz == 0;
      const bool masked = !zero_f && g.nyquist == 0 && nnz >= 2 && (q.z != 0.f || nyqz);
      float n1 = 0.f, n2 = 0.f, n3 = 0.f;
      if (!zero_f) {
        const float x1 = q.x, x2 = q.y, x3 = mz * g.inv_lz;
        const float inv = rsqrtf(x1 * x1 + x2 * x2 + x3 * x3);
        n1 = x1 * inv;
        n2 = x2 * inv;
        n3 = x3 * inv;
      }
      const float2 a0 = v[0][k2], a1 = v[1][k2], a2 = v[2][k2];
      float2 p1, p2, p3;   // this half's share of v = tau_hat n
      if (h == 0) {
        p1 = make_float2(a0.x * n1, a0.y * n1);
        p2 = make_float2(a1.x * n2, a1.y * n2);
        p3 = make_float2(a2.x * n3, a2.y * n3);
      } else {
        p1 = make_float2(a2.x * n2 + a1.x * n3, a2.y * n2 + a1.y * n3);
        p2 = make_float2(a2.x * n1 + a0.x * n3, a2.y * n1 + a0.y * n3);
        p3 = make_float2(a1.x * n1 + a0.x * n2, a1.y * n1 + a0.y * n2);
      }
      p1.x += __shfl_xor_sync(0xffffffffu, p1.x, 16);
      p1.y += __shfl_xor_sync(0xffffffffu, p1.y, 16);
      p2.x += __shfl_xor_sync(0xffffffffu, p2.x, 16);
      p2.y += __shfl_xor_sync(0xffffffffu, p2.y, 16);
      p3.x += __shfl_xor_sync(0xffffffffu, p3.x, 16);
      p3.y += __shfl_xor_sync(0xffffffffu, p3.y, 16);
      const float sx = n1 * p1.x + n2 * p2.x + n3 * p3.x;
      const float sy = n1 * p1.y + n2 * p2.y + n3 * p3.y;
      const float2 w1 = make_float2((p1.x - ga.a * n1 * sx) * ga.inv_mu0,
                                    (p1.y - ga.a * n1 * sy) * ga.inv_mu0);
      const float2 w2 = make_float2((p2.x - ga.a * n2 * sx) * ga.inv_mu0,
                                    (p2.y - ga.a * n2 * sy) * ga.inv_mu0);
      const float2 w3 = make_float2((p3.x - ga.a * n3 * sx) * ga.inv_mu0,
                                    (p3.y - ga.a * n3 * sy) * ga.inv_mu0);
      float2 o0, o1, o2;
      if (h == 0) {
        o0 = make_float2(-n1 * w1.x, -n1 * w1.y);
        o1 = make_float2(-n2 * w2.x, -n2 * w2.y);
        o2 = make_float2(-n3 * w3.x, -n3 * w3.y);
      } else {
        o0 = make_float2(-0.5f * (n2 * w3.x + n3 * w2.x), -0.5f * (n2 * w3.y + n3 * w2.y));
        o1 = make_float2(-0.5f * (n1 * w3.x + n3 * w1.x), -0.5f * (n1 * w3.y + n3 * w1.y));
        o2 = make_float2(-0.5f * (n1 * w2.x + n2 * w1.x), -0.5f * (n1 * w2.y + n2 * w1.y));
      }
      if (zero_f) {
        const bool full = mode == GM_FULL_MAP;
        o0 = make_float2(full ? ga.En[3 * h] : 0.f, 0.f);
        o1 = make_float2(full ? ga.En[3 * h + 1] : 0.f, 0.f);
        o2 = make_float2(full ? ga.En[3 * h + 2] : 0.f, 0.f);
      } else if (masked) {
        o0 = o1 = o2 = make_float2(0.f, 0.f);
      }
      v[0][k2] = o0;
      v[1][k2] = o1;
      v[2][k2] = o2;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      RegDft<Z2, true>::run(v[j]);
#pragma unroll
      for (int n2 = 1; n2 < Z2; ++n2) v[j][n2] = cmulc(v[j][n2], twz[n2 * Z1 + k1]);
      float2* p = B + ((3 * h + j) * T + t) * NZP + k1 * Z2;
#pragma unroll
      for (int i = 0; i < Z2; ++i) p[i] = v[j][i];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 6 * T * Z2; q += blockDim.x) {   // inverse step 2 -> global
    const int t = q % T, c = (q / T) % 6, n2 = q / (6 * T);
    const int m = m0 + t;
    const float2* p = B + (c * T + t) * NZP + n2;
    float2 v[Z1];
#pragma unroll
    for (int i = 0; i < Z1; ++i) v[i] = p[i * Z2];
    RegDft<Z1, true>::run(v);
    if (m < plane) {
      float2* dst = spec + ((size_t)c * NZ + n2) * plane + m;
      const size_t zs = (size_t)Z2 * plane;
#pragma unroll
      for (int i = 0; i < Z1; ++i) dst[i * zs] = v[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Five-pass variant for planes that do not fit in shared memory (nx = 256)
// and for nx != ny: rows along x, pencils along y, the z pass above, pencils
// along y (inverse), rows along x (inverse).  The spectrum layout and slot
// orders are those of the three-pass path, so pass B is shared.
// ---------------------------------------------------------------------------
constexpr int kRows = 32;             // rows per block in the inverse x pass
constexpr int kRowsP = kRows + 1;     // odd stride

// Forward x pass of the five-pass variant, one block per (component group,
// group of kRowsG rows, z): group 0 holds the three normal components, group 1
// the three shear components, as 3 kRowsG lines.  Each strain component is
// loaded once and the trace once per voxel (Eq. 2.3), then the packed
// half-length x-FFT and the real-to-complex untangling run on all lines.
constexpr int kRowsG = 16;              // rows of one component per block
constexpr int kLinesG = 3 * kRowsG;     // lines per block (three components)
constexpr int kLinesGP = kLinesG + 1;   // odd stride

template <int NX>
__global__ void __launch_bounds__(kThreads) k_rows_fwd(GridDev g, const float* __restrict__ in,
                                                       float2* __restrict__ spec, int mode) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  extern __shared__ float2 sm[];
  float2* P = sm;                                  // [SX][kLinesGP], line = j kRowsG + row
  float2* twx = P + SX * kLinesGP;
  float2* r2c = twx + NXH;
  float2* dm = r2c + SX;
  const int grp = blockIdx.x, y0 = blockIdx.y * kRowsG, z = blockIdx.z;
  const int ny = g.ny;
  for (int i = threadIdx.x; i < NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) dm[i] = g.dmat[i];
  __syncthreads();
  const size_t n2 = (size_t)g.n / 2;
  const size_t row2 = ((size_t)z * ny + y0) * NXH;         // float2 offset of row y0
  const float2* in2 = reinterpret_cast<const float2*>(in) + 3 * grp * n2 + row2;
  const uchar2* ph2 = reinterpret_cast<const uchar2*>(g.phase) + row2;
  // Loads are issued in groups of U voxel pairs per thread before any use.
  constexpr int TOT = kRowsG * NXH, U = 2;
  for (int base = threadIdx.x; base < TOT; base += U * kThreads) {
    float2 e[U][3];
    uchar2 ph[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kThreads;
      if (idx < TOT && y0 + idx / NXH < ny) {
#pragma unroll
        for (int j = 0; j < 3; ++j) e[u][j] = in2[j * n2 + idx];
        if (mode != GM_RAW_TAU) ph[u] = ph2[idx];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * kThreads;
      if (idx < TOT) {
        const int r = idx / NXH, h = idx - r * NXH;
        float2 t[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) t[j] = make_float2(0.f, 0.f);
        if (y0 + r < ny) {
          if (mode == GM_RAW_TAU) {
#pragma unroll
            for (int j = 0; j < 3; ++j) t[j] = e[u][j];
          } else {
            const float2 d0 = dm[ph[u].x], d1 = dm[ph[u].y];
#pragma unroll
            for (int j = 0; j < 3; ++j)
              t[j] = make_float2(2.f * d0.y * e[u][j].x, 2.f * d1.y * e[u][j].y);
            if (grp == 0) {
              const float trx = e[u][0].x + e[u][1].x + e[u][2].x;
              const float try_ = e[u][0].y + e[u][1].y + e[u][2].y;
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                t[j].x = fmaf(d0.x, trx, t[j].x);
                t[j].y = fmaf(d1.x, try_, t[j].y);
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) P[h * kLinesGP + j * kRowsG + r] = t[j];
      }
    }
  }
  __syncthreads();
  smem_fft<NXH, false, kLinesG, 1, kLinesGP>(P, twx);
  for (int t = threadIdx.x; t < kLinesG * (NXH / 2 + 1); t += blockDim.x) {
    const int r = t % kLinesG, k = t / kLinesG;
    if (k == 0) {
      const float2 z0 = P[r];
      P[r] = make_float2(z0.x + z0.y, 0.f);
      P[NXH * kLinesGP + r] = make_float2(z0.x - z0.y, 0.f);
    } else {
      const int kk = NXH - k;
      const int sk = slot_of<NXH>(k), skk = slot_of<NXH>(kk);
      const float2 a = P[sk * kLinesGP + r], b = P[skk * kLinesGP + r];
      P[sk * kLinesGP + r] = r2c_post(a, b, r2c[k]);
      if (kk != k) P[skk * kLinesGP + r] = r2c_post(b, a, r2c[kk]);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kLinesG * SX; idx += blockDim.x) {
    const int l = idx / SX, sx = idx - l * SX;
    const int j = l / kRowsG, r = l - j * kRowsG;
    if (y0 + r < ny)
      spec[((size_t)(3 * grp + j) * g.nz + z) * g.plane + (size_t)(y0 + r) * SX + sx] =
          P[sx * kLinesGP + l];
  }
}

template <int NX>
__global__ void __launch_bounds__(kThreads) k_rows_inv(GridDev g, const float2* __restrict__ spec,
                                                       float* __restrict__ outp, float scale) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  extern __shared__ float2 sm[];
  float2* P = sm;
  float2* twx = P + SX * kRowsP;
  float2* r2c = twx + NXH;
  const int c = blockIdx.x, y0 = blockIdx.y * kRows, z = blockIdx.z;
  const int ny = g.ny;
  for (int i = threadIdx.x; i < NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  const float2* src = spec + ((size_t)c * g.nz + z) * g.plane + (size_t)y0 * SX;
  for (int idx = threadIdx.x; idx < kRows * SX; idx += blockDim.x) {
    const int r = idx / SX, sx = idx - r * SX;
    P[sx * kRowsP + r] = (y0 + r < ny) ? src[idx] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kRows * (NXH / 2 + 1); t += blockDim.x) {
    const int r = t % kRows, k = t / kRows;
    if (k == 0) {
      P[r] = c2r_pre(P[r], P[NXH * kRowsP + r], make_float2(1.f, 0.f));
    } else {
      const int kk = NXH - k;
      const int sk = slot_of<NXH>(k), skk = slot_of<NXH>(kk);
      const float2 a = P[sk * kRowsP + r], b = P[skk * kRowsP + r];
      P[sk * kRowsP + r] = c2r_pre(a, b, r2c[k]);
      if (kk != k) P[skk * kRowsP + r] = c2r_pre(b, a, r2c[kk]);
    }
  }
  __syncthreads();
  smem_fft<NXH, true, kRows, 1, kRowsP>(P, twx);
  const size_t n2 = (size_t)g.n / 2;
  float2* out2 = reinterpret_cast<float2*>(outp) + c * n2 + ((size_t)z * ny + y0) * NXH;
  for (int idx = threadIdx.x; idx < kRows * NXH; idx += blockDim.x) {
    const int r = idx / NXH, h = idx - r * NXH;
    if (y0 + r < ny) out2[idx] = cscale(P[h * kRowsP + r], scale);
  }
}

// The inverse x-row pass of the five-pass variant with the tangling fused
// into x step 1 and x step 2 writing the real rows straight to global memory
// (nx/2 with a two-step split and an even first factor).  Rows past ny are
// skipped.  (A forward counterpart -- strain rows read in x step 1, untangling
// fused into x step 2 -- measured slower than k_rows_fwd at 256^3: 280 against
// 248 us.)
template <int NX>
__global__ void __launch_bounds__(kThreads) k_rows_inv_direct(GridDev g, const float2* __restrict__ spec,
                                                              float* __restrict__ outp, float scale) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  constexpr int X1 = Split<NXH>::N1, X2 = Split<NXH>::N2;
  static_assert(X2 > 1 && X1 % 2 == 0, "x split must have two steps and an even first factor");
  extern __shared__ float2 sm[];
  float2* P = sm;                                  // [SX][kRowsP]
  float2* twx = P + SX * kRowsP;
  float2* r2c = twx + NXH;
  const int c = blockIdx.x, y0 = blockIdx.y * kRows, z = blockIdx.z;
  const int ny = g.ny;
  allow_dependent_launch();
  for (int i = threadIdx.x; i < NXH; i += blockDim.x) twx[i] = g.tw_x[i];
  for (int i = threadIdx.x; i < SX; i += blockDim.x) r2c[i] = g.r2c_w[i];
  grid_dependency_wait();
  const float2* src = spec + ((size_t)c * g.nz + z) * g.plane + (size_t)y0 * SX;
  for (int idx = threadIdx.x; idx < kRows * SX; idx += blockDim.x) {
    const int r = idx / SX, sx = idx - r * SX;
    P[sx * kRowsP + r] = (y0 + r < ny) ? src[idx] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  constexpr int NU = X1 / 2 + 1;   // tangling fused into x step 1 (inverse)
  constexpr int LS = kRowsP;
  for (int t = threadIdx.x; t < kRows * NU; t += blockDim.x) {
    const int b = t % kRows, u = t / kRows;
    float2* p = P + b;
    if (u == 0 || u == X1 / 2) {
      const int k1 = u;
      float2 v[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) v[i] = p[(k1 * X2 + i) * LS];
      float2 o[X2];
      if (k1 == 0) {
        o[0] = c2r_pre(v[0], p[NXH * LS], make_float2(1.f, 0.f));
#pragma unroll
        for (int i = 1; i < X2; ++i) {
          const int ip = X2 - i;
          if (i < ip) {
            o[i] = c2r_pre(v[i], v[ip], r2c[X1 * i]);
            o[ip] = c2r_pre(v[ip], v[i], r2c[X1 * ip]);
          } else if (i == ip) {
            o[i] = c2r_pre(v[i], v[i], r2c[X1 * i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < X2; ++i) {
          const int ip = X2 - 1 - i;
          if (i < ip) {
            o[i] = c2r_pre(v[i], v[ip], r2c[X1 / 2 + X1 * i]);
            o[ip] = c2r_pre(v[ip], v[i], r2c[X1 / 2 + X1 * ip]);
          } else if (i == ip) {
            o[i] = c2r_pre(v[i], v[i], r2c[X1 / 2 + X1 * i]);
          }
        }
      }
      RegDft<X2, true>::run(o);
#pragma unroll
      for (int n2 = 1; n2 < X2; ++n2) o[n2] = cmulc(o[n2], twx[n2 * X1 + k1]);
#pragma unroll
      for (int i = 0; i < X2; ++i) p[(k1 * X2 + i) * LS] = o[i];
    } else {
      const int k1 = u, k1p = X1 - u;
      float2 va[X2], vb[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        va[i] = p[(k1 * X2 + i) * LS];
        vb[i] = p[(k1p * X2 + i) * LS];
      }
      float2 oa[X2], ob[X2];
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        const int ip = X2 - 1 - i;
        oa[i] = c2r_pre(va[i], vb[ip], r2c[k1 + X1 * i]);
        ob[ip] = c2r_pre(vb[ip], va[i], r2c[k1p + X1 * ip]);
      }
      RegDft<X2, true>::run(oa);
      RegDft<X2, true>::run(ob);
#pragma unroll
      for (int n2 = 1; n2 < X2; ++n2) {
        oa[n2] = cmulc(oa[n2], twx[n2 * X1 + k1]);
        ob[n2] = cmulc(ob[n2], twx[n2 * X1 + k1p]);
      }
#pragma unroll
      for (int i = 0; i < X2; ++i) {
        p[(k1 * X2 + i) * LS] = oa[i];
        p[(k1p * X2 + i) * LS] = ob[i];
      }
    }
  }
  __syncthreads();
  const size_t nf2 = (size_t)g.n / 2;
  float2* out2 = reinterpret_cast<float2*>(outp) + c * nf2 + ((size_t)z * ny + y0) * NXH;
  for (int q = threadIdx.x; q < kRows * X2; q += blockDim.x) {   // x step 2 -> global
    int r, n2;
    row_task<X2, kRows>(q, r, n2);
    float2 v[X1];
#pragma unroll
    for (int i = 0; i < X1; ++i) v[i] = P[(n2 + X2 * i) * kRowsP + r];
    RegDft<X1, true>::run(v);
    if (y0 + r < ny) {
      float2* o = out2 + (size_t)r * NXH + n2;
#pragma unroll
      for (int i = 0; i < X1; ++i) o[i * X2] = cscale(v[i], scale);
    }
  }
}

// In-place FFT along y of TY consecutive x slots of one (component, z) plane.
template <int NY>
struct YPencilCfg {
  static constexpr int TY = NY >= 256 ? 16 : (NY >= 128 ? 32 : 64);
  static constexpr int NYP = NY + 1;
};

template <int NY, bool INV>
__global__ void __launch_bounds__(kThreads) k_ypencil(GridDev g, float2* __restrict__ spec) {
  using C = YPencilCfg<NY>;
  constexpr int TY = C::TY, NYP = C::NYP;
  extern __shared__ float2 sm[];
  float2* B = sm;                  // [TY][NYP]
  float2* twy = B + TY * NYP;
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  const int sx0 = blockIdx.x * TY;
  const int SX = g.nxh + 1;
  float2* pl = spec + (size_t)blockIdx.y * g.plane;     // blockIdx.y = c * nz + z
  for (int idx = threadIdx.x; idx < TY * NY; idx += blockDim.x) {
    const int t = idx % TY, y = idx / TY;
    B[t * NYP + y] = (sx0 + t < SX) ? pl[(size_t)y * SX + sx0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  smem_fft<NY, INV, TY, NYP, 1>(B, twy);
  for (int idx = threadIdx.x; idx < TY * NY; idx += blockDim.x) {
    const int t = idx % TY, y = idx / TY;
    if (sx0 + t < SX) pl[(size_t)y * SX + sx0 + t] = B[t * NYP + y];
  }
}

// The y pass of the five-pass variant with its outer FFT steps on global
// memory: the first register step reads the TY columns straight from the
// spectrum, the second writes them straight back, and shared memory holds the
// exchange between the two steps only (column stride NY + 1: conflict-free).
template <int NY, bool INV>
__global__ void __launch_bounds__(kThreads) k_ypencil_direct(GridDev g, float2* __restrict__ spec) {
  using C = YPencilCfg<NY>;
  constexpr int TY = C::TY, NYP = C::NYP;
  constexpr int Y1 = Split<NY>::N1, Y2 = Split<NY>::N2;
  static_assert(Y2 > 1, "two register steps");
  extern __shared__ __align__(16) float2 sm[];
  float2* B = sm;                  // [TY][NYP]
  float2* twy = B + TY * NYP;
  allow_dependent_launch();
  for (int i = threadIdx.x; i < NY; i += blockDim.x) twy[i] = g.tw_y[i];
  grid_dependency_wait();
  __syncthreads();
  const int sx0 = blockIdx.x * TY;
  const int SX = g.nxh + 1;
  float2* pl = spec + (size_t)blockIdx.y * g.plane;     // blockIdx.y = c * nz + z
  if (!INV) {
    for (int q = threadIdx.x; q < TY * Y2; q += blockDim.x) {   // step 1: Y1-point, stride Y2
      const int t = q % TY, n2 = q / TY;
      const bool ok = sx0 + t < SX;
      float2 v[Y1];
#pragma unroll
      for (int i = 0; i < Y1; ++i)
        v[i] = ok ? pl[(size_t)(n2 + Y2 * i) * SX + sx0 + t] : make_float2(0.f, 0.f);
      RegDft<Y1, false>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < Y1; ++k1) v[k1] = cmul(v[k1], twy[n2 * Y1 + k1]);
#pragma unroll
      for (int i = 0; i < Y1; ++i) B[t * NYP + n2 + Y2 * i] = v[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TY * Y1; q += blockDim.x) {   // step 2: Y2-point, contiguous
      const int t = q % TY, k1 = q / TY;
      float2 v[Y2];
#pragma unroll
      for (int i = 0; i < Y2; ++i) v[i] = B[t * NYP + k1 * Y2 + i];
      RegDft<Y2, false>::run(v);
      if (sx0 + t < SX) {
#pragma unroll
        for (int i = 0; i < Y2; ++i) pl[(size_t)(k1 * Y2 + i) * SX + sx0 + t] = v[i];
      }
    }
  } else {
    for (int q = threadIdx.x; q < TY * Y1; q += blockDim.x) {   // inverse step 1
      const int t = q % TY, k1 = q / TY;
      const bool ok = sx0 + t < SX;
      float2 v[Y2];
#pragma unroll
      for (int i = 0; i < Y2; ++i)
        v[i] = ok ? pl[(size_t)(k1 * Y2 + i) * SX + sx0 + t] : make_float2(0.f, 0.f);
      RegDft<Y2, true>::run(v);
#pragma unroll
      for (int n2 = 1; n2 < Y2; ++n2) v[n2] = cmulc(v[n2], twy[n2 * Y1 + k1]);
#pragma unroll
      for (int i = 0; i < Y2; ++i) B[t * NYP + k1 * Y2 + i] = v[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TY * Y2; q += blockDim.x) {   // inverse step 2
      const int t = q % TY, n2 = q / TY;
      float2 v[Y1];
#pragma unroll
      for (int i = 0; i < Y1; ++i) v[i] = B[t * NYP + n2 + Y2 * i];
      RegDft<Y1, true>::run(v);
      if (sx0 + t < SX) {
#pragma unroll
        for (int i = 0; i < Y1; ++i) pl[(size_t)(n2 + Y2 * i) * SX + sx0 + t] = v[i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int NX>
static cudaError_t launch_plane_passes(const GridDev& g, const float* in, float* out,
                                       float2* spec, int mode, int which, cudaStream_t st) {
  using C = PlaneCfg<NX, NX>;
  const dim3 grid(6, g.nz);
  if (which == 0) {
    const size_t smem = (size_t)(C::PLANE_F2 + C::TAB_F2 + 256) * sizeof(float2);
    cudaError_t e = set_smem(k_pass_a<NX, NX>, smem);
    if (e != cudaSuccess) return e;
    k_pass_a<NX, NX><<<grid, kPlaneThreads, smem, st>>>(g, in, spec, mode);
  } else {
    const size_t smem = (size_t)(C::PLANE_F2 + C::TAB_F2) * sizeof(float2);
    cudaError_t e = set_smem(k_pass_c<NX, NX>, smem);
    if (e != cudaSuccess) return e;
    k_pass_c<NX, NX><<<grid, kPlaneThreads, smem, st>>>(g, spec, out, 1.0f / (float)g.n);
  }
  return cudaGetLastError();
}

template <int NZ, int TT>
static cudaError_t launch_pencil_tile(const GridDev& g, float2* spec, int mode,
                                      const GammaArgs& ga, cudaStream_t st) {
  using C = PencilCfg<NZ, TT>;
  const size_t smem = (size_t)(6 * C::T * C::NZP + NZ) * sizeof(float2);
  if (TT < 1 || smem > 227 * 1024) return cudaErrorInvalidValue;   // variant not available
  const int blocks = (g.plane + C::T - 1) / C::T;
  cudaError_t e;
  if constexpr (NZ >= 256 && C::T >= 8) {
    if ((e = set_smem(k_pass_b_wide<NZ, TT>, smem)) != cudaSuccess) return e;
    k_pass_b_wide<NZ, TT><<<blocks, 2 * kThreads, smem, st>>>(g, spec, mode, ga);
  } else {
    if ((e = set_smem(k_pass_b<NZ, TT>, smem)) != cudaSuccess) return e;
    k_pass_b<NZ, TT><<<blocks, kThreads, smem, st>>>(g, spec, mode, ga);
  }
  return cudaGetLastError();
}

template <int NZ>
static cudaError_t launch_pencil_pass(const GridDev& g, float2* spec, int mode, const GammaArgs& ga,
                                      cudaStream_t st) {
  constexpr int T0 = PencilCfg<NZ>::T;
  switch (g.pencil_t) {
    case 1: return launch_pencil_tile<NZ, (T0 / 2 > 0 ? T0 / 2 : 1)>(g, spec, mode, ga, st);
    case 2: return launch_pencil_tile<NZ, 2 * T0>(g, spec, mode, ga, st);
    default: return launch_pencil_tile<NZ, T0>(g, spec, mode, ga, st);
  }
}


template <int NX>
static cudaError_t launch_rows(const GridDev& g, const float* in, float* out, float2* spec,
                               int mode, int which, cudaStream_t st) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  const dim3 grid(6, (g.ny + kRows - 1) / kRows, g.nz);
  if constexpr (Split<NXH>::N2 > 1 && Split<NXH>::N1 % 2 == 0) {
    if (which == 1) {
      const size_t smem = (size_t)(SX * kRowsP + NXH + SX) * sizeof(float2);
      cudaError_t e;
      if ((e = set_smem(k_rows_inv_direct<NX>, smem)) != cudaSuccess) return e;
      return launch_pdl(k_rows_inv_direct<NX>, grid, kThreads, smem, st, g, (const float2*)spec,
                        out, 1.0f / (float)g.n);
    }
  }
  if (which == 0) {
    const dim3 grid_f(2, (g.ny + kRowsG - 1) / kRowsG, g.nz);
    const size_t smem = (size_t)(SX * kLinesGP + NXH + SX + 256) * sizeof(float2);
    cudaError_t e = set_smem(k_rows_fwd<NX>, smem);
    if (e != cudaSuccess) return e;
    k_rows_fwd<NX><<<grid_f, kThreads, smem, st>>>(g, in, spec, mode);
  } else {
    const size_t smem = (size_t)(SX * kRowsP + NXH + SX) * sizeof(float2);
    cudaError_t e = set_smem(k_rows_inv<NX>, smem);
    if (e != cudaSuccess) return e;
    k_rows_inv<NX><<<grid, kThreads, smem, st>>>(g, spec, out, 1.0f / (float)g.n);
  }
  return cudaGetLastError();
}

template <int NY>
static cudaError_t launch_ypencil(const GridDev& g, float2* spec, bool inv, cudaStream_t st) {
  using C = YPencilCfg<NY>;
  const size_t smem = (size_t)(C::TY * C::NYP + NY) * sizeof(float2);
  const dim3 grid((g.nxh + 1 + C::TY - 1) / C::TY, 6 * g.nz);
  cudaError_t e;
  if constexpr (Split<NY>::N2 > 1) {
    if (inv) {
      if ((e = set_smem(k_ypencil_direct<NY, true>, smem)) != cudaSuccess) return e;
      return launch_pdl(k_ypencil_direct<NY, true>, grid, kThreads, smem, st, g, spec);
    }
    if ((e = set_smem(k_ypencil_direct<NY, false>, smem)) != cudaSuccess) return e;
    return launch_pdl(k_ypencil_direct<NY, false>, grid, kThreads, smem, st, g, spec);
  }
  if (inv) {
    if ((e = set_smem(k_ypencil<NY, true>, smem)) != cudaSuccess) return e;
    k_ypencil<NY, true><<<grid, kThreads, smem, st>>>(g, spec);
  } else {
    if ((e = set_smem(k_ypencil<NY, false>, smem)) != cudaSuccess) return e;
    k_ypencil<NY, false><<<grid, kThreads, smem, st>>>(g, spec);
  }
  return cudaGetLastError();
}


// the fused plane passes: nx = ny with a two-step x split of nx/2 and an even
// first factor; the fused pencil pass: 128 / split_n1(nz) pencils per block
#define RPM_FUSED_PLANE_SIZES(X) X(48) X(64) X(96) X(128)
// (nz = 64 takes the 8-pencil tile of the original z pass: 0.0293 vs
// 0.0314 ms per 64^3 apply)
#define RPM_FUSED_Z_SIZES(X) X(32) X(48) X(96) X(128)

template <int NX>
static cudaError_t launch_fused_plane(const GridDev& g, const float* in, float* out, float2* spec,
                                      int mode, int which, cudaStream_t st,
                                      const float* add = nullptr) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  const size_t tab = (size_t)(NXH + NX + SX) * sizeof(float2);
  const size_t smem = (size_t)NX * SX * sizeof(float2) + tab;
  cudaError_t e;
  if (which == 0) {
    if ((e = set_smem(k_plane_fwd<NX, NX>, smem + 256 * sizeof(float2))) != cudaSuccess) return e;
    return launch_pdl(k_plane_fwd<NX, NX>, dim3(6, g.nz), kPlaneThreads,
                      smem + 256 * sizeof(float2), st, g, in, spec, mode);
  }
  if ((e = set_smem(k_plane_inv<NX, NX, false>, smem)) != cudaSuccess) return e;
  return launch_pdl(k_plane_inv<NX, NX, false>, dim3(6 * g.nz), kPlaneThreads, smem, st, g,
                    (const float2*)spec, out, 1.0f / (float)g.n, add, (const float4*)nullptr);
}

// pass C with Algorithm 3's post-step (clusters of three blocks)
template <int NX>
static cudaError_t launch_fused_inv_post(const GridDev& g, float* out, float2* spec,
                                         const float* eps, const float4* post, cudaStream_t st) {
  constexpr int NXH = NX / 2, SX = NXH + 1;
  constexpr int F2 = NX * SX + NXH + NX + SX;
  const size_t smem = (size_t)(F2 + (F2 & 1)) * sizeof(float2) + 256 * sizeof(float4);
  cudaError_t e;
  if ((e = set_smem(k_plane_inv<NX, NX, true>, smem)) != cudaSuccess) return e;
  return launch_pdl_cluster(k_plane_inv<NX, NX, true>, dim3(6 * g.nz), kPlaneThreads, smem, st,
                            3u, g, (const float2*)spec, out, 1.0f / (float)g.n, eps, post);
}

template <int NZ>
static cudaError_t launch_fused_pencil(const GridDev& g, float2* spec, int mode,
                                       const GammaArgs& ga, cudaStream_t st) {
  using C = PencilFused<NZ>;
  const size_t smem = (size_t)(6 * C::T * C::NZP + NZ) * sizeof(float2);
  cudaError_t e;
  if ((e = set_smem(k_pencil_green<NZ>, smem)) != cudaSuccess) return e;
  return launch_pdl(k_pencil_green<NZ>, dim3((g.plane + C::T - 1) / C::T), kThreads, smem, st, g,
                    spec, mode, ga);
}

static bool fused_plane_ok(const GridDev& g, const float2* spec) {
  if (g.nx != g.ny || ((uintptr_t)spec & 15) != 0) return false;   // pass C's bulk copy
  switch (g.nx) {
#define RPM_CASE(N) case N:
    RPM_FUSED_PLANE_SIZES(RPM_CASE)
#undef RPM_CASE
    return true;
    default: return false;
  }
}

static bool fused_pencil_ok(int nz) {
  switch (nz) {
#define RPM_CASE(N) case N:
    RPM_FUSED_Z_SIZES(RPM_CASE)
#undef RPM_CASE
    return true;
    default: return false;
  }
}

static cudaError_t dispatch_fused_plane(const GridDev& g, const float* in, float* out,
                                        float2* spec, int mode, int which, cudaStream_t st,
                                        const float* add = nullptr) {
  switch (g.nx) {
#define RPM_CASE(N) \
  case N: return launch_fused_plane<N>(g, in, out, spec, mode, which, st, add);
    RPM_FUSED_PLANE_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch_fused_inv_post(const GridDev& g, float* out, float2* spec,
                                           const float* eps, const float4* post, cudaStream_t st) {
  switch (g.nx) {
#define RPM_CASE(N) \
  case N: return launch_fused_inv_post<N>(g, out, spec, eps, post, st);
    RPM_FUSED_PLANE_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch_fused_pencil(const GridDev& g, float2* spec, int mode,
                                         const GammaArgs& ga, cudaStream_t st) {
  switch (g.nz) {
#define RPM_CASE(N) \
  case N: return launch_fused_pencil<N>(g, spec, mode, ga, st);
    RPM_FUSED_Z_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

#define RPM_SIZES(X) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(256)
#define RPM_Z_SIZES(X) \
  X(1) X(2) X(3) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(256)

static cudaError_t dispatch_rows(const GridDev& g, const float* in, float* out, float2* spec,
                                 int mode, int which, cudaStream_t st) {
  switch (g.nx) {
#define RPM_CASE(N) \
  case N: return launch_rows<N>(g, in, out, spec, mode, which, st);
    RPM_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch_ypencil(const GridDev& g, float2* spec, bool inv, cudaStream_t st) {
  switch (g.ny) {
#define RPM_CASE(N) \
  case N: return launch_ypencil<N>(g, spec, inv, st);
    RPM_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

// three-pass (whole xy planes in shared memory) when the plane fits
static bool plane_fits(int nx, int ny) { return nx == ny && nx <= 128; }

static bool xy_size_ok(int n) {
  switch (n) {
#define RPM_CASE(N) case N:
    RPM_SIZES(RPM_CASE)
#undef RPM_CASE
    return true;
    default: return false;
  }
}

static bool z_size_ok(int n) {
  switch (n) {
#define RPM_CASE(N) case N:
    RPM_Z_SIZES(RPM_CASE)
#undef RPM_CASE
    return true;
    default: return false;
  }
}

#define RPM_PLANE_SIZES(X) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128)

static cudaError_t dispatch_plane(const GridDev& g, const float* in, float* out, float2* spec,
                                  int mode, int which, cudaStream_t st) {
  switch (g.nx) {
#define RPM_CASE(N) \
  case N: return launch_plane_passes<N>(g, in, out, spec, mode, which, st);
    RPM_PLANE_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t dispatch_pencil(const GridDev& g, float2* spec, int mode, const GammaArgs& ga,
                                   cudaStream_t st) {
  switch (g.nz) {
#define RPM_CASE(N) \
  case N: return launch_pencil_pass<N>(g, spec, mode, ga, st);
    RPM_Z_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return cudaErrorInvalidValue;
  }
}

// The plane kernels g.plane_v resolves to on this grid: 0 fused, 1 whole-plane, 2 five-pass.
static int plane_path(const GridDev& g, const float2* spec) {
  if (g.plane_v == 0 && fused_plane_ok(g, spec)) return 0;
  if (g.plane_v <= 1 && plane_fits(g.nx, g.ny)) return 1;
  return 2;
}

static bool fused_z(const GridDev& g) { return g.pencil_t == 0 && fused_pencil_ok(g.nz); }

bool fused_z_pass(const GridDev& g) { return fused_z(g); }

// (for a spectrum buffer from cudaMalloc, whose alignment is 256 bytes)
int plane_variant(const GridDev& g) { return plane_path(g, nullptr); }

int gamma_launches(const GridDev& g) { return plane_variant(g) == 2 ? 5 : 3; }

int pencil_tile(const GridDev& g) {
  if (fused_z(g)) return 128 / split_n1(g.nz);
  int t0;
  switch (g.nz) {
#define RPM_CASE(N) \
  case N: t0 = PencilCfg<N>::T; break;
    RPM_Z_SIZES(RPM_CASE)
#undef RPM_CASE
    default: return 0;
  }
  return g.pencil_t == 1 ? (t0 / 2 > 0 ? t0 / 2 : 1) : (g.pencil_t == 2 ? 2 * t0 : t0);
}


bool grid_supported(int nx, int ny, int nz) {
  return xy_size_ok(nx) && xy_size_ok(ny) && z_size_ok(nz);
}

static GammaArgs gamma_args(const GridDev& g, const double E[6]) {
  GammaArgs ga;
  for (int c = 0; c < 6; ++c) ga.En[c] = (float)(E ? E[c] * (double)g.n : 0.0);
  const double l0 = g.lam0, m0 = g.mu0;
  ga.a = (float)((l0 + m0) / (l0 + 2.0 * m0));
  ga.inv_mu0 = (float)(1.0 / m0);
  return ga;
}

static cudaError_t z_pass(const GridDev& g, float2* spec, int mode, const GammaArgs& ga,
                          cudaStream_t st) {
  return fused_z(g) ? dispatch_fused_pencil(g, spec, mode, ga, st)
                    : dispatch_pencil(g, spec, mode, ga, st);
}

// the post-step rides on the fused plane passes; fields are read as float2
static bool fused_post_ok(const GridDev& g, const float* in, const float* out,
                          const float2* spec) {
  return plane_path(g, spec) == 0 && ((uintptr_t)in & 7) == 0 && ((uintptr_t)out & 7) == 0;
}

int polarization_launches(const GridDev& g, const float* in, const float* out,
                          const float2* spec) {
  return fused_post_ok(g, in, out, spec) ? 3 : gamma_launches(g) + 1;
}

cudaError_t launch_polarization_map(const GridDev& g, const float4* post, const float* in,
                                    float* eb, float* out, float2* spec, const double Eb[6],
                                    int mode, cudaStream_t st) {
  cudaError_t e;
  if (fused_post_ok(g, in, out, spec)) {
    const GammaArgs ga = gamma_args(g, Eb);
    if ((e = dispatch_fused_plane(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
    if ((e = z_pass(g, spec, mode, ga, st)) != cudaSuccess) return e;
    return dispatch_fused_inv_post(g, out, spec, in, post, st);
  }
  if ((e = launch_apply_gamma(g, in, eb, spec, Eb, mode, st)) != cudaSuccess) return e;
  return launch_polarization_post(g, post, in, eb, out, st);
}

// the added field rides on the fused last pass (float2 accesses)
static bool fused_add_ok(const GridDev& g, const float* out, const float* add,
                         const float2* spec) {
  return plane_path(g, spec) == 0 && ((uintptr_t)out & 7) == 0 && ((uintptr_t)add & 7) == 0;
}

int gamma_add_launches(const GridDev& g, const float* out, const float* add, const float2* spec) {
  return gamma_launches(g) + (add && !fused_add_ok(g, out, add, spec) ? 1 : 0);
}

cudaError_t launch_apply_gamma(const GridDev& g, const float* in, float* out, float2* spec,
                               const double E[6], int mode, cudaStream_t st, const float* add) {
  const GammaArgs ga = gamma_args(g, E);
  cudaError_t e;
  auto zpass = [&]() { return z_pass(g, spec, mode, ga, st); };
  const int path = plane_path(g, spec);
  if (path == 0 && (!add || fused_add_ok(g, out, add, spec))) {
    if ((e = dispatch_fused_plane(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
    if ((e = zpass()) != cudaSuccess) return e;
    return dispatch_fused_plane(g, in, out, spec, mode, 1, st, add);
  }
  if (path <= 1 && plane_fits(g.nx, g.ny)) {
    if ((e = dispatch_plane(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
    if ((e = zpass()) != cudaSuccess) return e;
    e = dispatch_plane(g, in, out, spec, mode, 1, st);
  } else {
    if ((e = dispatch_rows(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
    if ((e = dispatch_ypencil(g, spec, false, st)) != cudaSuccess) return e;
    if ((e = zpass()) != cudaSuccess) return e;
    if ((e = dispatch_ypencil(g, spec, true, st)) != cudaSuccess) return e;
    e = dispatch_rows(g, in, out, spec, mode, 1, st);
  }
  if (e != cudaSuccess || !add) return e;
  return launch_axpby(out, 1.f, out, 1.f, add, g.n, st);
}

}  // namespace rpm
