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
// The Green operator of the isotropic reference medium is evaluated on the
// fly from the unit wave vector n = xi/|xi|:
//   Gamma0_hat : tau_hat = sym(n (x) w),  w = (v - a n (n.v)) / mu0,
//   v = tau_hat n,  a = (lam0 + mu0) / (lam0 + 2 mu0),
// obtained from div(C0 : eps(u) + tau) = 0 in Fourier space.
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
// for the length (8 pencils = 64-byte rows at nz >= 128); the tile autotuner
// of rpm_create also tries half and twice the default (GridDev::pencil_t).
template <int NZ, int TT = 0>
struct PencilCfg {
  static constexpr int T = TT ? TT : (NZ >= 128 ? 8 : (NZ >= 64 ? 16 : 32));
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
  {
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
  }
  __syncthreads();
  smem_fft<NZ, false, 6 * T, NZP, 1>(B, twz);
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
      const float inv = 1.f / sqrtf(x1 * x1 + x2 * x2 + x3 * x3);
      green_apply(tv, x1 * inv, x2 * inv, x3 * inv, ga.a, ga.inv_mu0);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) B[(c * T + t) * NZP + sz] = tv[c];
  }
  __syncthreads();
  smem_fft<NZ, true, 6 * T, NZP, 1>(B, twz);
  for (int idx = threadIdx.x; idx < 6 * NZ * T; idx += blockDim.x) {
    const int t = idx % T, r = idx / T, z = r % NZ, c = r / NZ;
    const int m = m0 + t;
    if (m < plane) spec[((size_t)c * NZ + z) * plane + m] = B[(c * T + t) * NZP + z];
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
  if (inv) {
    if ((e = set_smem(k_ypencil<NY, true>, smem)) != cudaSuccess) return e;
    k_ypencil<NY, true><<<grid, kThreads, smem, st>>>(g, spec);
  } else {
    if ((e = set_smem(k_ypencil<NY, false>, smem)) != cudaSuccess) return e;
    k_ypencil<NY, false><<<grid, kThreads, smem, st>>>(g, spec);
  }
  return cudaGetLastError();
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

int gamma_launches(int nx, int ny) { return plane_fits(nx, ny) ? 3 : 5; }

int pencil_tile(const GridDev& g) {
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

cudaError_t launch_apply_gamma(const GridDev& g, const float* in, float* out, float2* spec,
                               const double E[6], int mode, cudaStream_t st) {
  GammaArgs ga;
  for (int c = 0; c < 6; ++c) ga.En[c] = (float)(E ? E[c] * (double)g.n : 0.0);
  const double l0 = g.lam0, m0 = g.mu0;
  ga.a = (float)((l0 + m0) / (l0 + 2.0 * m0));
  ga.inv_mu0 = (float)(1.0 / m0);
  cudaError_t e;
  if (plane_fits(g.nx, g.ny)) {
    if ((e = dispatch_plane(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
    if ((e = dispatch_pencil(g, spec, mode, ga, st)) != cudaSuccess) return e;
    return dispatch_plane(g, in, out, spec, mode, 1, st);
  }
  if ((e = dispatch_rows(g, in, out, spec, mode, 0, st)) != cudaSuccess) return e;
  if ((e = dispatch_ypencil(g, spec, false, st)) != cudaSuccess) return e;
  if ((e = dispatch_pencil(g, spec, mode, ga, st)) != cudaSuccess) return e;
  if ((e = dispatch_ypencil(g, spec, true, st)) != cudaSuccess) return e;
  return dispatch_rows(g, in, out, spec, mode, 1, st);
}

}  // namespace rpm
