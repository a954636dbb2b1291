// Learned warm start: a 3D spectral neural operator (truncated-Fourier layers),
// forward, backward and Adam, as declared in include/rpm_fno.h.
//
// One Fourier layer on B samples of W = 16 channels over an N^3 grid runs as
// three kernels:
//   k_xy_fwd    block per (z, b): for each channel, the x transform of the
//               plane restricted to kx < m, then the y transform restricted to
//               the 2m kept ky; writes the [ncol = 2m * m][W] mode columns of
//               the plane.
//   k_spec_fwd  block per (kept (ky, kx) column, sample): z transform to the
//               2m kept kz, complex channel mixing with the column's R (held
//               in shared memory), inverse z transform.  The backward
//               (k_spec_bwd) loops over the batch in one block per column so
//               that the R gradient is summed without atomics.
//   k_inv_xy    block per (y chunk, z, b): inverse y then inverse x transform
//               of the 16 channels, fused with the pointwise branch
//               A v + a and the activation (forward) or with the accumulation
//               of the input gradient (backward).
// The transforms are truncated DFTs (sums over the N points for each kept
// frequency, twiddles from one table of N roots): with m = 12 kept modes of
// N = 64 points the truncated sums cost about what a full FFT would and
// produce only the coefficients that are used.
//
// Parameter gradients of the pointwise maps (P, A_l, Q and biases) are
// outer-product sums over all voxels: each block accumulates them over tiles
// of 256 voxels staged in shared memory and writes one partial row; a second
// kernel adds the rows in a fixed order (float64), so gradients are
// deterministic.  Gradients of R_l are accumulated by the block that owns the
// (ky, kx) column, over the batch, in registers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "rpm.h"
#include "rpm_fno.h"
#include "rpm_internal.h"

namespace {

constexpr int W = RPM_FNO_WIDTH;   // channels of the hidden layers
constexpr int CV = 2;              // voxel features (the network's input channels)
constexpr int CE = 6;              // macroscopic strain components
constexpr int COUT = 6;            // strain components out
constexpr int NH = COUT * CE;      // localisation channels H[o][j]
constexpr int kMaxModes = RPM_FNO_MAX_MODES;
constexpr int kThreads = 256;
constexpr int kHeader = 768;       // floats before layer 0 in the parameter vector
constexpr int kLayerHead = W * W + W;
constexpr int kPwBlocksMax = 4 * 152;
constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)

// offsets of the head parameters
constexpr int kOffP = 0;
constexpr int kNeP = W * CV + W;                 // gradient entries of (P, p): 48
constexpr int kOffQ = kNeP;
constexpr int kNeA = W * W + W;                  // (A, a)
constexpr int kNeQ = NH * W + NH;                // (Q, q): 612
constexpr int kNeHead = kNeQ + 1;                // + squared-error sum
static_assert(kOffQ + kNeQ <= kHeader, "head parameters overflow the header");

size_t r_floats(int m) { return (size_t)2 * (2 * m * m) * (2 * m) * W * W; }
size_t layer_floats(int m) { return kLayerHead + r_floats(m); }
size_t layer_off(int m, int l) { return kHeader + (size_t)l * layer_floats(m); }

__device__ __forceinline__ int kfreq(int i, int m, int N) { return i < m ? i : N - 2 * m + i; }

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + tanhf(kGeluC * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(kGeluC * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * kGeluC * (1.f + 3.f * 0.044715f * x * x);
}

// ---------------------------------------------------------------------------
// Transforms
// ---------------------------------------------------------------------------

// k_xy_fwd: channels are transformed G at a time (G planes in shared memory,
// row-major with a row stride of N + 4 floats, an odd number of 16-byte
// units, so 16-byte reads of consecutive rows hit distinct banks).  Both
// stages are register-tiled truncated DFTs:
//   x stage  X_c[y][kx] = sum_x v_c[y][x] Tx[x][kx]     tile 4 rows (y, y + N/4,
//                                                        y + N/2, y + 3N/4) x 4 kx
//   y stage  V_c[ky][kx] = sum_y X_c[y][kx] Ty[y][ky]    tile 4 ky x 2 kx
// with twiddle tables Tx[x][kx] = exp(-2 pi i kx x / N) (kx padded to a
// multiple of 4 with zeros) and Ty[y][ky_i] likewise for the kept ky.
__host__ __device__ inline int xy_group(int N) { return N <= 64 ? 4 : 1; }
__host__ __device__ inline int pad4(int v) { return (v + 3) / 4 * 4; }
size_t xy_smem(int N, int m) {
  const size_t G = xy_group(N), NP = N + 4, MP = pad4(m), KP = pad4(2 * m);
  return (G * N * NP + 2 * (G * N * MP + N * MP + N * KP)) * 4;
}

// src [B][W][N][N][N] -> dst [B][N(z)][ncol][W] (complex); column = ky_i * m + kx.
// tw[j] = exp(-2 pi i j / N).
__global__ void __launch_bounds__(kThreads) k_xy_fwd(const float* __restrict__ src,
                                                     float2* __restrict__ dst,
                                                     const float2* __restrict__ twg, int N, int m) {
  extern __shared__ float4 smem4[];
  const int G = xy_group(N), NP = N + 4, MP = pad4(m), KP = pad4(2 * m);
  const int ncol = 2 * m * m;
  float* planeT = (float*)smem4;                       // [G][y][NP]
  float2* X = (float2*)(planeT + (size_t)G * N * NP);  // [G][y][MP]
  float2* Tx = X + (size_t)G * N * MP;                 // [x][MP]
  float2* Ty = Tx + N * MP;                            // [y][KP]
  const int tid = threadIdx.x, z = blockIdx.x, b = blockIdx.y;
  const long long NN = (long long)N * N;
  float2* d = dst + ((long long)b * N + z) * ncol * W;
  for (int i = tid; i < N * MP; i += kThreads) {
    const int x = i / MP, k = i - x * MP;
    Tx[i] = k < m ? twg[(k * x) % N] : make_float2(0.f, 0.f);
  }
  for (int i = tid; i < N * KP; i += kThreads) {
    const int y = i / KP, k = i - y * KP;
    Ty[i] = k < 2 * m ? twg[(kfreq(k, m, N) * y) % N] : make_float2(0.f, 0.f);
  }
  const int xq = N / 4, xk = MP / 4;          // x-stage tiles per channel: xq * xk
  const int yk = KP / 4, yx = MP / 2;         // y-stage tiles per channel: yk * yx
  for (int c0 = 0; c0 < W; c0 += G) {
    __syncthreads();   // previous group's readers are done
    for (int i = tid; i < G * N * N / 4; i += kThreads) {
      const int g = i / (N * N / 4), r = i - g * (N * N / 4);
      const int y = r / (N / 4), x = 4 * (r - y * (N / 4));
      *reinterpret_cast<float4*>(planeT + ((size_t)g * N + y) * NP + x) =
          *reinterpret_cast<const float4*>(
              src + (((long long)b * W + c0 + g) * N + z) * NN + (long long)y * N + x);
    }
    __syncthreads();
    for (int item = tid; item < G * xq * xk; item += kThreads) {
      const int g = item / (xq * xk), r = item - g * (xq * xk);
      const int yq = r / xk, kg = r - yq * xk;
      const float* pv = planeT + ((size_t)g * N + yq) * NP;   // rows yq + a N/4
      const float2* pt = Tx + 4 * kg;
      const int rs = xq * NP;                                 // N/4 rows apart
      float re[4][4], im[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) re[a][k] = im[a][k] = 0.f;
      for (int x = 0; x < N; x += 4) {
        float vv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float4 v = *reinterpret_cast<const float4*>(pv + a * rs + x);
          vv[a][0] = v.x;
          vv[a][1] = v.y;
          vv[a][2] = v.z;
          vv[a][3] = v.w;
        }
#pragma unroll
        for (int dx = 0; dx < 4; ++dx) {
          const float4 t01 = *reinterpret_cast<const float4*>(pt + (x + dx) * MP);
          const float4 t23 = *reinterpret_cast<const float4*>(pt + (x + dx) * MP + 2);
          const float tr[4] = {t01.x, t01.z, t23.x, t23.z};
          const float ti[4] = {t01.y, t01.w, t23.y, t23.w};
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              re[a][k] = fmaf(vv[a][dx], tr[k], re[a][k]);
              im[a][k] = fmaf(vv[a][dx], ti[k], im[a][k]);
            }
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        float2* px = X + ((size_t)g * N + yq + a * xq) * MP + 4 * kg;
#pragma unroll
        for (int k = 0; k < 4; ++k) px[k] = make_float2(re[a][k], im[a][k]);
      }
    }
    __syncthreads();
    for (int item = tid; item < G * yk * yx; item += kThreads) {
      const int g = item / (yk * yx), r = item - g * (yk * yx);
      const int kq = r / yx, kp = r - kq * yx;
      const float2* px = X + (size_t)g * N * MP + 2 * kp;
      const float2* pt = Ty + 4 * kq;
      float re[4][2], im[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) re[a][k] = im[a][k] = 0.f;
      for (int y = 0; y < N; ++y) {
        const float4 xv = *reinterpret_cast<const float4*>(px + y * MP);
        const float4 t01 = *reinterpret_cast<const float4*>(pt + y * KP);
        const float4 t23 = *reinterpret_cast<const float4*>(pt + y * KP + 2);
        const float xr[2] = {xv.x, xv.z}, xi[2] = {xv.y, xv.w};
        const float tr[4] = {t01.x, t01.z, t23.x, t23.z};
        const float ti[4] = {t01.y, t01.w, t23.y, t23.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            re[a][k] = fmaf(xr[k], tr[a], fmaf(-xi[k], ti[a], re[a][k]));
            im[a][k] = fmaf(xr[k], ti[a], fmaf(xi[k], tr[a], im[a][k]));
          }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int kyi = 4 * kq + a, kx = 2 * kp + k;
          if (kyi < 2 * m && kx < m)
            d[(kyi * m + kx) * W + c0 + g] = make_float2(re[a][k], im[a][k]);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of k_xy_fwd (configuration precision RPM_FNO_BF16): both
// truncated DFT stages as BF16 matrix products with float32 accumulation
// (mma.sync m16n8k16), operands staged in shared memory as bfloat16 and
// loaded with ldmatrix.
//   x stage  C[y][2kx + {re, im}] = sum_x v[y][x] (Tx_re, Tx_im)[x][kx]
//            M = N rows, K = N, Nout = 2 * round4(m)
//   y stage  D[r][kx] = sum_{y, re/im} Ay[r][2y + .] X[y][kx].(re, im), with
//            rows r < KPY giving Re V[ky_r] (Ty_re, -Ty_im) and rows KPY + r
//            giving Im V[ky_r] (Ty_im, Ty_re); M = 2 KPY, K = 2N, Nout = round8(m)
// Needs N % 16 == 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}
// D += A (16 x 16, row) * B (16 x 8, col), bfloat16 in, float32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

__host__ __device__ inline int round_up(int v, int q) { return (v + q - 1) / q * q; }

struct XyTc {
  int G, NPB, NX2, KPY, MY, MPY, KPB;
  __host__ __device__ XyTc(int N, int m) {
    G = N <= 64 ? 4 : 1;
    NPB = N + 8;                 // bf16 row stride of the staged planes (16-byte rows)
    NX2 = 2 * round_up(m, 4);    // x-stage output columns
    KPY = round_up(2 * m, 8);    // kept ky rows per part
    MY = 2 * KPY;
    MPY = round_up(m, 8);        // y-stage output columns (kx)
    KPB = 2 * N + 8;             // bf16 row stride of Ay and XT
  }
  __host__ __device__ size_t bytes(int N) const {
    return (size_t)2 * ((size_t)G * N * NPB + (size_t)NX2 * NPB + (size_t)MY * KPB +
                        (size_t)G * MPY * KPB) +
           (size_t)4 * G * MY * MPY;
  }
};
size_t xy_tc_smem(int N, int m) { return XyTc(N, m).bytes(N); }

// Templated on the grid side so that the index arithmetic divides by constants.
template <int N>
__global__ void __launch_bounds__(kThreads, 2) k_xy_fwd_tc(const float* __restrict__ src,
                                                        float2* __restrict__ dst,
                                                        const float2* __restrict__ twg, int m) {
  extern __shared__ float4 smem4[];
  const XyTc c(N, m);
  const int ncol = 2 * m * m;
  uint16_t* planes = reinterpret_cast<uint16_t*>(smem4);          // [G][N][NPB]
  uint16_t* BTx = planes + (size_t)c.G * N * c.NPB;                // [NX2][NPB]
  uint16_t* Ay = BTx + (size_t)c.NX2 * c.NPB;                      // [MY][KPB]
  uint16_t* XT = Ay + (size_t)c.MY * c.KPB;                        // [G][MPY][KPB]
  float* Ds = reinterpret_cast<float*>(XT + (size_t)c.G * c.MPY * c.KPB);   // [G][MY][MPY]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int z = blockIdx.x, b = blockIdx.y;
  const long long NN = (long long)N * N;
  float2* d = dst + ((long long)b * N + z) * ncol * W;
  for (int i = tid; i < c.NX2 * N; i += kThreads) {
    const int r = i / N, x = i - r * N, kx = r >> 1;
    float v = 0.f;
    if (kx < m) {
      const float2 t = twg[(kx * x) % N];
      v = (r & 1) ? t.y : t.x;
    }
    BTx[r * c.NPB + x] = bf16_bits(v);
  }
  for (int i = tid; i < c.KPY * N; i += kThreads) {
    const int r = i / N, y = i - r * N;
    float tr = 0.f, ti = 0.f;
    if (r < 2 * m) {
      const float2 t = twg[(kfreq(r, m, N) * y) % N];
      tr = t.x;
      ti = t.y;
    }
    uint16_t* re = Ay + (size_t)r * c.KPB + 2 * y;
    uint16_t* im = Ay + (size_t)(c.KPY + r) * c.KPB + 2 * y;
    re[0] = bf16_bits(tr);
    re[1] = bf16_bits(-ti);
    im[0] = bf16_bits(ti);
    im[1] = bf16_bits(tr);
  }
  const int nmt = N / 16, nnt = c.NX2 / 8;          // x-stage tiles per channel
  const int ymt = c.MY / 16, ynt = c.MPY / 8;        // y-stage tiles per channel
  for (int c0 = 0; c0 < W; c0 += c.G) {
    __syncthreads();   // tables written; the previous group's readers are done
    for (int i = tid; i < c.G * N * N / 4; i += kThreads) {
      const int g = i / (N * N / 4), r = i - g * (N * N / 4);
      const int y = r / (N / 4), x = 4 * (r - y * (N / 4));
      const float4 v = *reinterpret_cast<const float4*>(
          src + (((long long)b * W + c0 + g) * N + z) * NN + (long long)y * N + x);
      uint2 pk;
      pk.x = bf16x2_bits(v.x, v.y);
      pk.y = bf16x2_bits(v.z, v.w);
      *reinterpret_cast<uint2*>(planes + ((size_t)g * N + y) * c.NPB + x) = pk;
    }
    __syncthreads();
    for (int tile = warp; tile < c.G * nmt * nnt; tile += kThreads / 32) {
      const int g = tile / (nmt * nnt), r = tile - g * (nmt * nnt);
      const int mt = r / nnt, nt = r - mt * nnt;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t* pa = planes + ((size_t)g * N + 16 * mt + (lane & 15)) * c.NPB + (lane >> 4) * 8;
      const uint16_t* pb = BTx + (size_t)(8 * nt + (lane & 7)) * c.NPB + ((lane >> 3) & 1) * 8;
      for (int k0 = 0; k0 < N; k0 += 16) {
        uint32_t a[4], bb[2];
        ldsm_x4(a, pa + k0);
        ldsm_x2(bb, pb + k0);
        mma_bf16(acc, a, bb);
      }
      // acc: rows y = 16 mt + lane/4 (and + 8), columns 2t, 2t + 1 = (re, im) of kx = 4 nt + t
      const int y = 16 * mt + (lane >> 2), kx = 4 * nt + (lane & 3);
      uint32_t* xt = reinterpret_cast<uint32_t*>(XT + ((size_t)g * c.MPY + kx) * c.KPB);
      xt[y] = bf16x2_bits(acc[0], acc[1]);
      xt[y + 8] = bf16x2_bits(acc[2], acc[3]);
    }
    __syncthreads();
    for (int tile = warp; tile < c.G * ymt * ynt; tile += kThreads / 32) {
      const int g = tile / (ymt * ynt), r = tile - g * (ymt * ynt);
      const int mt = r / ynt, nt = r - mt * ynt;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t* pa = Ay + (size_t)(16 * mt + (lane & 15)) * c.KPB + (lane >> 4) * 8;
      const uint16_t* pb = XT + ((size_t)g * c.MPY + 8 * nt + (lane & 7)) * c.KPB +
                           ((lane >> 3) & 1) * 8;
      for (int k0 = 0; k0 < 2 * N; k0 += 16) {
        uint32_t a[4], bb[2];
        ldsm_x4(a, pa + k0);
        ldsm_x2(bb, pb + k0);
        mma_bf16(acc, a, bb);
      }
      float* ds = Ds + ((size_t)g * c.MY + 16 * mt + (lane >> 2)) * c.MPY + 8 * nt + 2 * (lane & 3);
      ds[0] = acc[0];
      ds[1] = acc[1];
      ds[8 * c.MPY] = acc[2];
      ds[8 * c.MPY + 1] = acc[3];
    }
    __syncthreads();
    for (int i = tid; i < c.G * 2 * m * m; i += kThreads) {
      const int g = i % c.G, col = i / c.G;
      const int kyi = col / m, kx = col - kyi * m;
      const float* ds = Ds + (size_t)g * c.MY * c.MPY;
      d[(long long)col * W + c0 + g] =
          make_float2(ds[kyi * c.MPY + kx], ds[(c.KPY + kyi) * c.MPY + kx]);
    }
  }
}

size_t spec_smem(int N, int m) {
  const size_t m2 = 2 * m;
  return (m2 * W * W + (size_t)N * W + 3 * m2 * W + N + (size_t)N * m2) * sizeof(float2);
}

// Tz[z][kz_i] = exp(-2 pi i kz z / N) for the kept kz (the inverse uses the conjugate).
__device__ __forceinline__ void z_table(const float2* twg, float2* Tz, int N, int m) {
  for (int i = threadIdx.x; i < N * 2 * m; i += kThreads) {
    const int z = i / (2 * m), k = i - z * (2 * m);
    Tz[i] = twg[(kfreq(k, m, N) * z) % N];
  }
}

// z transform of the column's [N][W] values to the 2m kept kz: out[kz_i][c].
__device__ __forceinline__ void z_dft(const float2* a, const float2* tw, float2* out, int N, int m,
                                      float scale) {
  for (int o = threadIdx.x; o < 2 * m * W; o += kThreads) {
    const int kzi = o / W, c = o % W;
    const int kz = kfreq(kzi, m, N);
    float re = 0.f, im = 0.f;
    int j = 0;
    for (int z = 0; z < N; ++z) {
      const float2 v = a[z * W + c], t = tw[j];
      re += v.x * t.x - v.y * t.y;
      im += v.x * t.y + v.y * t.x;
      j += kz;
      if (j >= N) j -= N;
    }
    out[o] = make_float2(scale * re, scale * im);
  }
}

// inverse z transform (no weights) of U[kz_i][c] to dst[z][c] (column stride given).
__device__ __forceinline__ void z_idft(const float2* U, const float2* Tz, float2* dst,
                                       long long zstride, int N, int m) {
  for (int o = threadIdx.x; o < N * W; o += kThreads) {
    const int z = o / W, c = o % W;
    float re = 0.f, im = 0.f;
    const float2* tz = Tz + z * 2 * m;
    for (int kzi = 0; kzi < 2 * m; ++kzi) {
      const float2 u = U[kzi * W + c], t = tz[kzi];
      re += u.x * t.x + u.y * t.y;   // u * conj(t)
      im += u.y * t.x - u.x * t.y;
    }
    dst[(long long)z * zstride + c] = make_float2(re, im);
  }
}

// A2 [B][N][ncol][W] -> V (saved, [ncol][B][2m][W]), U = V R, Bz [B][N][ncol][W].
__global__ void __launch_bounds__(kThreads) k_spec_fwd(const float2* __restrict__ A2,
                                                       const float2* __restrict__ R,
                                                       float2* __restrict__ Vs,
                                                       float2* __restrict__ Bz,
                                                       const float2* __restrict__ twg, int N, int m,
                                                       int B) {
  extern __shared__ float4 smem4[];
  const int m2 = 2 * m, ncol = 2 * m * m, col = blockIdx.x, tid = threadIdx.x;
  float2* Rs = (float2*)smem4;      // [kz_i][i][o]
  float2* a = Rs + m2 * W * W;      // [z][c]
  float2* V = a + N * W;            // [kz_i][c]
  float2* U = V + m2 * W;
  float2* tw = U + 2 * m2 * W;
  float2* Tz = tw + N;
  const int b = blockIdx.y;   // one sample per block
  const float4* r4 = (const float4*)(R + (long long)col * m2 * W * W);
  for (int i = tid; i < m2 * W * W / 2; i += kThreads) ((float4*)Rs)[i] = r4[i];
  for (int i = tid; i < N; i += kThreads) tw[i] = twg[i];
  z_table(twg, Tz, N, m);
  for (int i = tid; i < N * W; i += kThreads)
    a[i] = A2[((long long)b * N + i / W) * ncol * W + col * W + i % W];
  __syncthreads();
  z_dft(a, tw, V, N, m, 1.f);
  __syncthreads();
  float2* vs = Vs + ((long long)col * B + b) * m2 * W;
  for (int o = tid; o < m2 * W; o += kThreads) {
    vs[o] = V[o];
    const int kzi = o / W, oc = o % W;
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float2 v = V[kzi * W + i], r = Rs[(kzi * W + i) * W + oc];
      re += v.x * r.x - v.y * r.y;
      im += v.x * r.y + v.y * r.x;
    }
    U[o] = make_float2(re, im);
  }
  __syncthreads();
  z_idft(U, Tz, Bz + (long long)b * N * ncol * W + col * W, (long long)ncol * W, N, m);
}

// Tensor-core form of k_spec_fwd (RPM_FNO_BF16, N % 16 == 0): one block per
// kept (ky, kx) column and all samples, in groups of 16.  Per sample, the z
// transform to the kept kz is a BF16 product (rows Re / Im of each kz, K = 2N
// over (z, re/im)); the channel mixing of each kz is a BF16 product over the
// group (M = 16 samples, K = 32 over (i, re/im), N = 32 over (o, re/im), the
// real form of the complex R[kz]); the inverse z transform is again a product
// (rows Re / Im of each z, K over (kz, re/im)).  float32 accumulation; the
// forward spectra V are kept in float32 for the backward pass.
template <int N>
struct SpecTc {
  int m2, KPZ, MZ, KZB, KIB, MB;
  __host__ __device__ SpecTc(int m) {
    m2 = 2 * m;
    KPZ = round_up(2 * m, 8);   // kz rows per part
    MZ = 2 * KPZ;
    KZB = 2 * N + 8;            // row stride of Az and BTa
    KIB = 2 * KPZ + 8;          // row stride of Ainv and BTU
    MB = 32 + 8;                // row stride of the mixing operand
  }
  __host__ __device__ size_t bytes() const {
    return (size_t)2 * ((size_t)MZ * KZB + (size_t)2 * N * KIB + (size_t)W * KZB +
                        (size_t)KPZ * 16 * MB + (size_t)16 * W * KIB) +
           (size_t)4 * ((size_t)MZ * 16 + (size_t)2 * N * 16);
  }
};
template <int N>
size_t spec_tc_smem(int m) { return SpecTc<N>(m).bytes(); }

template <int N>
__global__ void __launch_bounds__(kThreads, 2) k_spec_fwd_tc(const float2* __restrict__ A2,
                                                          const float2* __restrict__ R,
                                                          float2* __restrict__ Vs,
                                                          float2* __restrict__ Bz,
                                                          const float2* __restrict__ twg, int m,
                                                          int B) {
  extern __shared__ float4 smem4[];
  const SpecTc<N> c(m);
  const int m2 = c.m2, ncol = 2 * m * m, col = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint16_t* Az = reinterpret_cast<uint16_t*>(smem4);       // [MZ][KZB]
  uint16_t* Ainv = Az + (size_t)c.MZ * c.KZB;                // [2N][KIB]
  uint16_t* BTa = Ainv + (size_t)2 * N * c.KIB;              // [W][KZB]
  uint16_t* Vm = BTa + (size_t)W * c.KZB;                    // [KPZ][16][MB]
  uint16_t* BTU = Vm + (size_t)c.KPZ * 16 * c.MB;            // [16][W][KIB]
  float* Dz = reinterpret_cast<float*>(BTU + (size_t)16 * W * c.KIB);   // [MZ][16]
  float* Di = Dz + c.MZ * 16;                                            // [2N][16]
  const float2* Rc = R + (long long)col * m2 * W * W;
  for (int i = tid; i < c.KPZ * N; i += kThreads) {
    const int r = i / N, z = i - r * N;
    float tr = 0.f, ti = 0.f;
    if (r < m2) {
      const float2 t = twg[(kfreq(r, m, N) * z) % N];
      tr = t.x;
      ti = t.y;
    }
    *reinterpret_cast<uint32_t*>(Az + (size_t)r * c.KZB + 2 * z) = bf16x2_bits(tr, -ti);
    *reinterpret_cast<uint32_t*>(Az + (size_t)(c.KPZ + r) * c.KZB + 2 * z) = bf16x2_bits(ti, tr);
    // inverse: row z (re) (Tr, Ti), row N + z (im) (-Ti, Tr) at column pair r
    *reinterpret_cast<uint32_t*>(Ainv + (size_t)z * c.KIB + 2 * r) = bf16x2_bits(tr, ti);
    *reinterpret_cast<uint32_t*>(Ainv + (size_t)(N + z) * c.KIB + 2 * r) = bf16x2_bits(-ti, tr);
  }
  const int zmt = c.MZ / 16, imt = 2 * N / 16;
  for (int g0 = 0; g0 < B; g0 += 16) {
    const int gb = min(16, B - g0);
    __syncthreads();   // tables written; the previous group's readers are done
    for (int i = tid; i < c.KPZ * 16 * c.MB / 2; i += kThreads)
      reinterpret_cast<uint32_t*>(Vm)[i] = 0u;
    for (int i = tid; i < 16 * W * c.KIB / 2; i += kThreads)
      reinterpret_cast<uint32_t*>(BTU)[i] = 0u;
    for (int bi = 0; bi < gb; ++bi) {
      const int b = g0 + bi;
      __syncthreads();   // BTa / Dz readers of the previous sample are done
      for (int i = tid; i < N * W; i += kThreads) {
        const int z = i / W, cc = i - z * W;
        const float2 a = A2[((long long)b * N + z) * ncol * W + col * W + cc];
        *reinterpret_cast<uint32_t*>(BTa + (size_t)cc * c.KZB + 2 * z) = bf16x2_bits(a.x, a.y);
      }
      __syncthreads();
      for (int tile = warp; tile < zmt * 2; tile += kThreads / 32) {
        const int mt = tile >> 1, nt = tile & 1;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const uint16_t* pa = Az + (size_t)(16 * mt + (lane & 15)) * c.KZB + (lane >> 4) * 8;
        const uint16_t* pb = BTa + (size_t)(8 * nt + (lane & 7)) * c.KZB + ((lane >> 3) & 1) * 8;
        for (int k0 = 0; k0 < 2 * N; k0 += 16) {
          uint32_t a[4], bb[2];
          ldsm_x4(a, pa + k0);
          ldsm_x2(bb, pb + k0);
          mma_bf16(acc, a, bb);
        }
        float* d = Dz + (16 * mt + (lane >> 2)) * 16 + 8 * nt + 2 * (lane & 3);
        d[0] = acc[0];
        d[1] = acc[1];
        d[8 * 16] = acc[2];
        d[8 * 16 + 1] = acc[3];
      }
      __syncthreads();
      float2* vs = Vs + ((long long)col * B + b) * m2 * W;
      for (int o = tid; o < m2 * W; o += kThreads) {
        const int kzi = o / W, cc = o - kzi * W;
        const float re = Dz[kzi * 16 + cc], im = Dz[(c.KPZ + kzi) * 16 + cc];
        vs[o] = make_float2(re, im);
        *reinterpret_cast<uint32_t*>(Vm + ((size_t)kzi * 16 + bi) * c.MB + 2 * cc) =
            bf16x2_bits(re, im);
      }
    }
    __syncthreads();
    // channel mixing per kz: U[b][(o, re/im)] = sum_(i, re/im) V[b][(i, re/im)] Rr[kz]
    for (int tile = warp; tile < m2 * 4; tile += kThreads / 32) {
      const int kzi = tile >> 2, nt = tile & 3;
      const float2* rk = Rc + (size_t)kzi * W * W;
      const int o = 4 * nt + ((lane >> 2) >> 1), ro = (lane >> 2) & 1;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t* pa = Vm + ((size_t)kzi * 16 + (lane & 15)) * c.MB + (lane >> 4) * 8;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t a[4], bb[2];
        ldsm_x4(a, pa + 16 * ks);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = 8 * ks + (lane & 3) + 4 * h;
          const float2 r = rk[i * W + o];
          bb[h] = ro ? bf16x2_bits(r.y, r.x) : bf16x2_bits(r.x, -r.y);
        }
        mma_bf16(acc, a, bb);
      }
      // rows b = lane/4 (+8), columns n = 8 nt + 2t (+1) = (o', re/im), o' = 4 nt + t
      const int oo = 4 * nt + (lane & 3);
      const int b0 = lane >> 2;
      *reinterpret_cast<uint32_t*>(BTU + ((size_t)b0 * W + oo) * c.KIB + 2 * kzi) =
          bf16x2_bits(acc[0], acc[1]);
      *reinterpret_cast<uint32_t*>(BTU + ((size_t)(b0 + 8) * W + oo) * c.KIB + 2 * kzi) =
          bf16x2_bits(acc[2], acc[3]);
    }
    for (int bi = 0; bi < gb; ++bi) {
      const int b = g0 + bi;
      __syncthreads();   // BTU complete; Di readers of the previous sample are done
      for (int tile = warp; tile < imt * 2; tile += kThreads / 32) {
        const int mt = tile >> 1, nt = tile & 1;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const uint16_t* pa = Ainv + (size_t)(16 * mt + (lane & 15)) * c.KIB + (lane >> 4) * 8;
        const uint16_t* pb = BTU + ((size_t)bi * W + 8 * nt + (lane & 7)) * c.KIB +
                             ((lane >> 3) & 1) * 8;
        for (int k0 = 0; k0 < 2 * c.KPZ; k0 += 16) {
          uint32_t a[4], bb[2];
          ldsm_x4(a, pa + k0);
          ldsm_x2(bb, pb + k0);
          mma_bf16(acc, a, bb);
        }
        float* d = Di + (16 * mt + (lane >> 2)) * 16 + 8 * nt + 2 * (lane & 3);
        d[0] = acc[0];
        d[1] = acc[1];
        d[8 * 16] = acc[2];
        d[8 * 16 + 1] = acc[3];
      }
      __syncthreads();
      float2* bz = Bz + (long long)b * N * ncol * W + col * W;
      for (int i = tid; i < N * W; i += kThreads) {
        const int z = i / W, oc = i - z * W;
        bz[(long long)z * ncol * W + oc] = make_float2(Di[z * 16 + oc], Di[(N + z) * 16 + oc]);
      }
    }
  }
}

// Backward of k_spec_fwd.  A2 holds the xy transform of dz; dU = w(kx) / N^3 *
// (z transform); gR[col] = sum_b dU conj(V); dV = sum_o dU conj(R); Bz = inverse z of dV.
__global__ void __launch_bounds__(kThreads) k_spec_bwd(const float2* __restrict__ A2,
                                                       const float2* __restrict__ R,
                                                       const float2* __restrict__ Vs,
                                                       float2* __restrict__ gR,
                                                       float2* __restrict__ Bz,
                                                       const float2* __restrict__ twg, int N, int m,
                                                       int B, float inv_n3) {
  extern __shared__ float4 smem4[];
  const int m2 = 2 * m, ncol = 2 * m * m, col = blockIdx.x, tid = threadIdx.x;
  float2* Rs = (float2*)smem4;
  float2* a = Rs + m2 * W * W;
  float2* dU = a + N * W;
  float2* V = dU + m2 * W;
  float2* dV = V + m2 * W;
  float2* tw = dV + m2 * W;
  float2* Tz = tw + N;
  const int kx = col % m;
  const float wgt = (kx == 0 ? 1.f : 2.f) * inv_n3;
  const float4* r4 = (const float4*)(R + (long long)col * m2 * W * W);
  for (int i = tid; i < m2 * W * W / 2; i += kThreads) ((float4*)Rs)[i] = r4[i];
  for (int i = tid; i < N; i += kThreads) tw[i] = twg[i];
  z_table(twg, Tz, N, m);
  const int gi = tid / W, go = tid % W;   // this thread's (i, o) entry of gR
  float2 g[2 * kMaxModes];
#pragma unroll
  for (int k = 0; k < 2 * kMaxModes; ++k) g[k] = make_float2(0.f, 0.f);
  for (int b = 0; b < B; ++b) {
    __syncthreads();
    for (int i = tid; i < N * W; i += kThreads)
      a[i] = A2[((long long)b * N + i / W) * ncol * W + col * W + i % W];
    const float2* vs = Vs + ((long long)col * B + b) * m2 * W;
    for (int o = tid; o < m2 * W; o += kThreads) V[o] = vs[o];
    __syncthreads();
    z_dft(a, tw, dU, N, m, wgt);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2 * kMaxModes; ++k)
      if (k < m2) {
        const float2 u = dU[k * W + go], v = V[k * W + gi];
        g[k].x += u.x * v.x + u.y * v.y;   // u * conj(v)
        g[k].y += u.y * v.x - u.x * v.y;
      }
    for (int o = tid; o < m2 * W; o += kThreads) {
      const int kzi = o / W, i = o % W;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int s = 0; s < W; ++s) {
        const int oc = (s + i) & (W - 1);   // rotated: conflict-free rows of Rs
        const float2 u = dU[kzi * W + oc], r = Rs[(kzi * W + i) * W + oc];
        re += u.x * r.x + u.y * r.y;        // u * conj(r)
        im += u.y * r.x - u.x * r.y;
      }
      dV[o] = make_float2(re, im);
    }
    __syncthreads();
    z_idft(dV, Tz, Bz + (long long)b * N * ncol * W + col * W, (long long)ncol * W, N, m);
  }
  float2* gr = gR + (long long)col * m2 * W * W;
#pragma unroll
  for (int k = 0; k < 2 * kMaxModes; ++k)
    if (k < m2) gr[k * W * W + tid] = g[k];
}

// k_inv_xy shared memory: S [ncol][W], Y [YC][m][W], TyT [2m][YC] (conjugate
// roots of rows y0..y0+YC-1), Txw [m][N] (weighted roots), then A and a.
size_t inv_smem(int m, int YC) {
  return ((size_t)2 * m * m * W + (size_t)YC * m * W + (size_t)2 * m * YC +
          (size_t)m * RPM_FNO_MAX_N) * sizeof(float2) + kLayerHead * sizeof(float);
}

// Pointwise end of k_inv_xy for the two voxels of a thread (at0, at1 =
// offsets of their channel 0); each row of A is loaded once for both.
template <bool BWD>
__device__ __forceinline__ void inv_pointwise(const float (&u0)[W], const float (&u1)[W],
                                              const float* Al, const float* __restrict__ vin,
                                              float* __restrict__ zsave, float* __restrict__ vout,
                                              long long at0, long long at1, long long N3,
                                              int last) {
  if constexpr (BWD) {   // all loads before any store: the stores cannot delay the loads
    float g0[W], g1[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      g0[c] = vout[at0 + c * N3];
      g1[c] = vout[at1 + c * N3];
    }
#pragma unroll
    for (int c = 0; c < W; ++c) {
      vout[at0 + c * N3] = g0[c] + u0[c];
      vout[at1 + c * N3] = g1[c] + u1[c];
    }
  } else {
    float v0[W], v1[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      v0[c] = vin[at0 + c * N3];
      v1[c] = vin[at1 + c * N3];
    }
#pragma unroll
    for (int oc = 0; oc < W; ++oc) {
      float s0 = Al[W * W + oc] + u0[oc], s1 = Al[W * W + oc] + u1[oc];
      const float4* ar = reinterpret_cast<const float4*>(Al + oc * W);
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const float4 av = ar[q];
        s0 = fmaf(av.x, v0[4 * q], fmaf(av.y, v0[4 * q + 1],
                  fmaf(av.z, v0[4 * q + 2], fmaf(av.w, v0[4 * q + 3], s0))));
        s1 = fmaf(av.x, v1[4 * q], fmaf(av.y, v1[4 * q + 1],
                  fmaf(av.z, v1[4 * q + 2], fmaf(av.w, v1[4 * q + 3], s1))));
      }
      if (last) {
        vout[at0 + oc * N3] = s0;
        vout[at1 + oc * N3] = s1;
      } else {
        zsave[at0 + oc * N3] = s0;
        zsave[at1 + oc * N3] = s1;
        vout[at0 + oc * N3] = gelu(s0);
        vout[at1 + oc * N3] = gelu(s1);
      }
    }
  }
}

// Inverse y and x transforms of the mode columns of plane (z, b), rows
// [y0, y0 + YC), fused with the pointwise part of the layer.
//   BWD = false: z = A v + a + u (u weighted c(kx) / N^3); writes zsave (unless
//                last) and vout = gelu(z) (z on the last layer).
//   BWD = true : vout += u (unweighted).
// y stage: Y[yy][kx][c] = sum_ky S[ky][kx][c] conj(root(ky y)), tile 4 rows x 2
// channels; x stage: u_c(x) = sum_kx w(kx) Re(Y[yy][kx][c] exp(+i 2 pi kx x / N))
// for the two voxels x and x + N/2 of a thread, then the pointwise map.
template <bool BWD>
__global__ void __launch_bounds__(kThreads, 2) k_inv_xy(const float2* __restrict__ Bz,
                                                     const float2* __restrict__ twg,
                                                     const float* __restrict__ layer,
                                                     const float* __restrict__ vin,
                                                     float* __restrict__ zsave,
                                                     float* __restrict__ vout, int N, int m,
                                                     int YC, int last, float inv_n3) {
  extern __shared__ float4 smem4[];
  const int ncol = 2 * m * m, tid = threadIdx.x, m2 = 2 * m;
  float2* S = (float2*)smem4;          // [ncol][W]
  float2* Y = S + ncol * W;            // [yy][kx][c]
  float2* TyT = Y + YC * m * W;        // [ky_i][yy]
  float2* Txw = TyT + m2 * YC;         // [kx][x]
  float* Al = (float*)(Txw + m * RPM_FNO_MAX_N);   // A [o][c], a [o]
  const int y0 = blockIdx.x * YC, z = blockIdx.y, b = blockIdx.z;
  const long long N3 = (long long)N * N * N;
  const float2* src = Bz + ((long long)b * N + z) * ncol * W;
  for (int i = tid; i < ncol * W / 2; i += kThreads) ((float4*)S)[i] = ((const float4*)src)[i];
  for (int i = tid; i < m2 * YC; i += kThreads) {
    const int k = i / YC, yy = i - k * YC;
    TyT[i] = twg[(kfreq(k, m, N) * (y0 + yy)) % N];
  }
  for (int i = tid; i < m * N; i += kThreads) {
    const int kx = i / N, x = i - kx * N;
    const float w = BWD ? 1.f : (kx == 0 ? inv_n3 : 2.f * inv_n3);
    const float2 t = twg[(kx * x) % N];
    Txw[i] = make_float2(w * t.x, w * t.y);
  }
  if (!BWD)
    for (int i = tid; i < kLayerHead; i += kThreads) Al[i] = layer[i];
  __syncthreads();
  const int nyq = YC / 4;
  for (int item = tid; item < nyq * m * (W / 2); item += kThreads) {
    const int yq = item / (m * (W / 2)), r = item - yq * (m * (W / 2));
    const int kx = r / (W / 2), cp = r - kx * (W / 2);
    float re[4][2], im[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 2; ++k) re[a][k] = im[a][k] = 0.f;
    for (int kyi = 0; kyi < m2; ++kyi) {
      const float4 sv = *reinterpret_cast<const float4*>(S + (kyi * m + kx) * W + 2 * cp);
      const float4 t01 = *reinterpret_cast<const float4*>(TyT + kyi * YC + 4 * yq);
      const float4 t23 = *reinterpret_cast<const float4*>(TyT + kyi * YC + 4 * yq + 2);
      const float sr[2] = {sv.x, sv.z}, si[2] = {sv.y, sv.w};
      const float tr[4] = {t01.x, t01.z, t23.x, t23.z};
      const float ti[4] = {t01.y, t01.w, t23.y, t23.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) {   // s * conj(t)
          re[a][k] = fmaf(sr[k], tr[a], fmaf(si[k], ti[a], re[a][k]));
          im[a][k] = fmaf(si[k], tr[a], fmaf(-sr[k], ti[a], im[a][k]));
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        Y[((4 * yq + a) * m + kx) * W + 2 * cp + k] = make_float2(re[a][k], im[a][k]);
  }
  __syncthreads();
  const int half = N / 2;
  for (int item = tid; item < YC * half; item += kThreads) {
    const int yy = item / half, x = item - yy * half;
    float u0[W], u1[W];
#pragma unroll
    for (int c = 0; c < W; ++c) u0[c] = u1[c] = 0.f;
    for (int kx = 0; kx < m; ++kx) {
      const float2 t0 = Txw[kx * N + x], t1 = Txw[kx * N + x + half];
      const float4* yr = reinterpret_cast<const float4*>(Y + (yy * m + kx) * W);
#pragma unroll
      for (int q = 0; q < W / 2; ++q) {
        const float4 yv = yr[q];   // channels 2q, 2q + 1
        u0[2 * q] = fmaf(yv.x, t0.x, fmaf(yv.y, t0.y, u0[2 * q]));
        u0[2 * q + 1] = fmaf(yv.z, t0.x, fmaf(yv.w, t0.y, u0[2 * q + 1]));
        u1[2 * q] = fmaf(yv.x, t1.x, fmaf(yv.y, t1.y, u1[2 * q]));
        u1[2 * q + 1] = fmaf(yv.z, t1.x, fmaf(yv.w, t1.y, u1[2 * q + 1]));
      }
    }
    const long long vox0 = ((long long)z * N + y0 + yy) * N + x;
    inv_pointwise<BWD>(u0, u1, Al, vin, zsave, vout, (long long)b * W * N3 + vox0,
                       (long long)b * W * N3 + vox0 + half, N3, last);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core form of k_inv_xy (RPM_FNO_BF16, N % 16 == 0).  Both inverse
// stages are BF16 matrix products with float32 accumulation:
//   y stage  D1[r][kx W + c] = sum_{kyi, re/im} A1[r][.] S[kyi][kx][c].(re, im),
//            rows r < YC giving Re Y[yy = r] (Ty_re, Ty_im) and rows YC + yy
//            giving Im Y (-Ty_im, Ty_re): M = 2 YC, K = round16(4m), Nout = m W
//   x stage  u[yy W + c][x] = sum_{kx, re/im} Y[yy][kx][c].(re, im) w(kx) (cos, -sin)
//            M = YC W, K = round16(2m), Nout = N
// Each warp stages the x-stage output of one row yy (16 channels x N voxels)
// in its own shared-memory slab and runs the pointwise end of the layer on
// those voxels (inv_pointwise, as in k_inv_xy).
// ---------------------------------------------------------------------------
struct InvTc {
  int K1, K1P, N1, M1, K2, K2P, UP, YC;
  __host__ __device__ InvTc(int N, int m, int yc) {
    YC = yc;
    K1 = round_up(4 * m, 16);
    K1P = K1 + 8;
    N1 = m * W;
    M1 = 2 * yc;
    K2 = round_up(2 * m, 16);
    K2P = K2 + 8;
    UP = N + 4;
  }
  __host__ __device__ size_t bytes(int N) const {
    return (size_t)2 * ((size_t)N1 * K1P + (size_t)M1 * K1P + (size_t)YC * W * K2P +
                        (size_t)N * K2P) +
           (size_t)4 * (8 * W * UP + kLayerHead);
  }
};
size_t inv_tc_smem(int N, int m, int YC) { return InvTc(N, m, YC).bytes(N); }

template <bool BWD, int N>
__global__ void __launch_bounds__(kThreads, 2) k_inv_xy_tc(const float2* __restrict__ Bz,
                                                        const float2* __restrict__ twg,
                                                        const float* __restrict__ layer,
                                                        const float* __restrict__ vin,
                                                        float* __restrict__ zsave,
                                                        float* __restrict__ vout, int m,
                                                        int YC, int last, float inv_n3) {
  extern __shared__ float4 smem4[];
  const InvTc c(N, m, YC);
  const int ncol = 2 * m * m, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint16_t* BT1 = reinterpret_cast<uint16_t*>(smem4);      // [N1][K1P]
  uint16_t* A1 = BT1 + (size_t)c.N1 * c.K1P;                 // [M1][K1P]
  uint16_t* A2 = A1 + (size_t)c.M1 * c.K1P;                  // [YC W][K2P]
  uint16_t* BT2 = A2 + (size_t)YC * W * c.K2P;               // [N][K2P]
  float* Uw = reinterpret_cast<float*>(BT2 + (size_t)N * c.K2P);   // [8][W][UP]
  float* Al = Uw + 8 * W * c.UP;
  const int y0 = blockIdx.x * YC, z = blockIdx.y, b = blockIdx.z;
  const long long N3 = (long long)N * N * N;
  const float2* src = Bz + ((long long)b * N + z) * ncol * W;
  for (int i = tid; i < ncol * W; i += kThreads) {
    const int cc = i % W, col = i / W;
    const int kyi = col / m, kx = col - kyi * m;
    const float2 sv = src[i];
    *reinterpret_cast<uint32_t*>(BT1 + (size_t)(kx * W + cc) * c.K1P + 2 * kyi) =
        bf16x2_bits(sv.x, sv.y);
  }
  const int pad1 = c.K1 - 4 * m;
  for (int i = tid; i < c.N1 * pad1; i += kThreads)
    BT1[(size_t)(i / pad1) * c.K1P + 4 * m + i % pad1] = 0;
  for (int i = tid; i < YC * (c.K1 / 2); i += kThreads) {
    const int yy = i / (c.K1 / 2), kyi = i - yy * (c.K1 / 2);
    float tr = 0.f, ti = 0.f;
    if (kyi < 2 * m) {
      const float2 t = twg[(kfreq(kyi, m, N) * (y0 + yy)) % N];
      tr = t.x;
      ti = t.y;
    }
    *reinterpret_cast<uint32_t*>(A1 + (size_t)yy * c.K1P + 2 * kyi) = bf16x2_bits(tr, ti);
    *reinterpret_cast<uint32_t*>(A1 + (size_t)(YC + yy) * c.K1P + 2 * kyi) = bf16x2_bits(-ti, tr);
  }
  const int pad2 = c.K2 - 2 * m;
  for (int i = tid; i < YC * W * pad2; i += kThreads)
    A2[(size_t)(i / pad2) * c.K2P + 2 * m + i % pad2] = 0;
  for (int i = tid; i < N * (c.K2 / 2); i += kThreads) {
    const int x = i / (c.K2 / 2), kx = i - x * (c.K2 / 2);
    float wr = 0.f, wi = 0.f;
    if (kx < m) {
      const float w = BWD ? 1.f : (kx == 0 ? inv_n3 : 2.f * inv_n3);
      const float2 t = twg[(kx * x) % N];
      wr = w * t.x;
      wi = w * t.y;
    }
    *reinterpret_cast<uint32_t*>(BT2 + (size_t)x * c.K2P + 2 * kx) = bf16x2_bits(wr, wi);
  }
  if (!BWD)
    for (int i = tid; i < kLayerHead; i += kThreads) Al[i] = layer[i];
  __syncthreads();
  const int nt1 = c.N1 / 8, mt1 = c.M1 / 16;
  for (int tile = warp; tile < mt1 * nt1; tile += kThreads / 32) {
    const int mt = tile / nt1, nt = tile - mt * nt1;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const uint16_t* pa = A1 + (size_t)(16 * mt + (lane & 15)) * c.K1P + (lane >> 4) * 8;
    const uint16_t* pb = BT1 + (size_t)(8 * nt + (lane & 7)) * c.K1P + ((lane >> 3) & 1) * 8;
    for (int k0 = 0; k0 < c.K1; k0 += 16) {
      uint32_t a[4], bb[2];
      ldsm_x4(a, pa + k0);
      ldsm_x2(bb, pb + k0);
      mma_bf16(acc, a, bb);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = 16 * mt + (lane >> 2) + 8 * h;
      const int part = r >= YC ? 1 : 0, yy = r - part * YC;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int n = 8 * nt + 2 * (lane & 3) + j;
        const int kx = n / W, cc = n - kx * W;
        A2[(size_t)(yy * W + cc) * c.K2P + 2 * kx + part] = bf16_bits(acc[2 * h + j]);
      }
    }
  }
  __syncthreads();
  float* uw = Uw + (size_t)warp * W * c.UP;
  const int half = N / 2;
  for (int mt = warp; mt < YC; mt += kThreads / 32) {   // one row yy = mt: its 16 channels
    for (int nt = 0; nt < N / 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t* pa = A2 + (size_t)(16 * mt + (lane & 15)) * c.K2P + (lane >> 4) * 8;
      const uint16_t* pb = BT2 + (size_t)(8 * nt + (lane & 7)) * c.K2P + ((lane >> 3) & 1) * 8;
      for (int k0 = 0; k0 < c.K2; k0 += 16) {
        uint32_t a[4], bb[2];
        ldsm_x4(a, pa + k0);
        ldsm_x2(bb, pb + k0);
        mma_bf16(acc, a, bb);
      }
      float* u = uw + (lane >> 2) * c.UP + 8 * nt + 2 * (lane & 3);
      u[0] = acc[0];
      u[1] = acc[1];
      u[8 * c.UP] = acc[2];
      u[8 * c.UP + 1] = acc[3];
    }
    __syncwarp();
#pragma unroll 1
    for (int x = lane; x < half; x += 32) {
      const long long at0 = (long long)b * W * N3 + ((long long)z * N + y0 + mt) * N + x;
      const long long at1 = at0 + half;
      const float* u0 = uw + x;
      const float* u1 = uw + x + half;
      if constexpr (BWD) {
        float g0[W], g1[W];
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
          g0[cc] = vout[at0 + cc * N3];
          g1[cc] = vout[at1 + cc * N3];
        }
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
          vout[at0 + cc * N3] = g0[cc] + u0[cc * c.UP];
          vout[at1 + cc * N3] = g1[cc] + u1[cc * c.UP];
        }
      } else {   // z = A v + a + u, then the activation (as inv_pointwise)
        float v0[W], v1[W];
#pragma unroll
        for (int cc = 0; cc < W; ++cc) {
          v0[cc] = vin[at0 + cc * N3];
          v1[cc] = vin[at1 + cc * N3];
        }
#pragma unroll 4
        for (int oc = 0; oc < W; ++oc) {
          float s0 = Al[W * W + oc] + u0[oc * c.UP], s1 = Al[W * W + oc] + u1[oc * c.UP];
          const float4* ar = reinterpret_cast<const float4*>(Al + oc * W);
#pragma unroll
          for (int q = 0; q < W / 4; ++q) {
            const float4 av = ar[q];
            s0 = fmaf(av.x, v0[4 * q], fmaf(av.y, v0[4 * q + 1],
                      fmaf(av.z, v0[4 * q + 2], fmaf(av.w, v0[4 * q + 3], s0))));
            s1 = fmaf(av.x, v1[4 * q], fmaf(av.y, v1[4 * q + 1],
                      fmaf(av.z, v1[4 * q + 2], fmaf(av.w, v1[4 * q + 3], s1))));
          }
          if (last) {
            vout[at0 + oc * N3] = s0;
            vout[at1 + oc * N3] = s1;
          } else {
            zsave[at0 + oc * N3] = s0;
            zsave[at1 + oc * N3] = s1;
            vout[at0 + oc * N3] = gelu(s0);
            vout[at1 + oc * N3] = gelu(s1);
          }
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Pointwise maps with parameter-gradient partial sums
// ---------------------------------------------------------------------------

// Per-block accumulation of sum_j L[a][j] R[b][j] (NA x NB) and sum_j L[a][j]
// over tiles of kThreads voxels staged in shared memory (row stride
// kThreads + 1: conflict-free column reads).
template <int NA, int NB>
struct TileAcc {
  static constexpr int NE = NA * NB + NA;
  static constexpr int PER = (NE + kThreads - 1) / kThreads;
  static constexpr int LD = kThreads + 1;
  float acc[PER];
  __device__ void init() {
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  }
  // all threads call this once per tile, after writing column threadIdx.x of sL / sR
  __device__ void step(const float* sL, const float* sR) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * kThreads;
      if (e < NA * NB) {
        const float* l = sL + (e / NB) * LD;
        const float* r = sR + (e % NB) * LD;
        float s = 0.f;
        for (int j = 0; j < kThreads; ++j) s = fmaf(l[j], r[j], s);
        acc[k] += s;
      } else if (e < NE) {
        const float* l = sL + (e - NA * NB) * LD;
        float s = 0.f;
        for (int j = 0; j < kThreads; ++j) s += l[j];
        acc[k] += s;
      }
    }
  }
  __device__ void store(float* part) const {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * kThreads;
      if (e < NE) part[e] = acc[k];
    }
  }
};

// Register-tiled variant for NA, NB multiples of 4: the tile is staged
// voxel-major (row j = voxel, stride LDL / LDR = 4 mod 8 floats, so that the
// 16-byte row writes of 8 consecutive threads hit distinct banks); a thread
// owns a 4 x 4 block of entries and every S-th voxel of the tile (2 x 16-byte
// loads per 16 FMA), and the S voxel slices are added in a fixed order at the
// end.  Row sums come with the b = 0 blocks.
template <int NA, int NB>
struct TileAcc4 {
  static_assert(NA % 4 == 0 && NB % 4 == 0, "4 x 4 entry blocks");
  static constexpr int LDL = (NA % 8 == 4) ? NA : NA + 4;
  static constexpr int LDR = (NB % 8 == 4) ? NB : NB + 4;
  static constexpr int TB = NB / 4, NT = (NA / 4) * TB;
  static constexpr int S = kThreads / NT;      // voxel slices
  static constexpr int NE = NA * NB + NA;
  static constexpr int SMEM = kThreads * (LDL + LDR);   // staging floats (>= S * NE)
  static_assert(S * NE <= SMEM, "slice reduction fits the staging area");
  float acc[4][4], rs[4];
  int ai, bi, sl;
  bool active;
  __device__ void init() {
    const int t = threadIdx.x;
    active = t < NT * S;
    const int tile = t % NT;
    sl = t / NT;
    ai = tile / TB;
    bi = tile - ai * TB;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      rs[x] = 0.f;
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    }
  }
  // all threads call this once per tile, after writing row threadIdx.x of sL / sR
  __device__ void step(const float* sL, const float* sR) {
    if (!active) return;
    for (int j = sl; j < kThreads; j += S) {
      const float4 l = *reinterpret_cast<const float4*>(sL + j * LDL + 4 * ai);
      const float4 r = *reinterpret_cast<const float4*>(sR + j * LDR + 4 * bi);
      const float lv[4] = {l.x, l.y, l.z, l.w}, rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        rs[x] += lv[x];
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(lv[x], rv[y], acc[x][y]);
      }
    }
  }
  // scratch: SMEM floats of shared memory no thread still reads (call after a barrier)
  __device__ void store(float* part, float* scratch) const {
    if (active) {
      float* sc = scratch + sl * NE;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
#pragma unroll
        for (int y = 0; y < 4; ++y) sc[(4 * ai + x) * NB + 4 * bi + y] = acc[x][y];
        if (bi == 0) sc[NA * NB + 4 * ai + x] = rs[x];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NE; e += kThreads) {
      float v = 0.f;
      for (int q = 0; q < S; ++q) v += scratch[q * NE + e];
      part[e] = v;
    }
  }
};

// v0 = P f + p.   total = B N^3 voxels.
__global__ void __launch_bounds__(kThreads) k_lift(const float* __restrict__ feat,
                                                   const float* __restrict__ prm,
                                                   float* __restrict__ v0, long long N3, int B) {
  __shared__ float Ps[kNeP];
  for (int i = threadIdx.x; i < kNeP; i += kThreads) Ps[i] = prm[kOffP + i];
  __syncthreads();
  const long long total = N3 * B;
  for (long long gidx = blockIdx.x * (long long)kThreads + threadIdx.x; gidx < total;
       gidx += (long long)gridDim.x * kThreads) {
    const int b = (int)(gidx / N3);
    const long long vox = gidx - b * N3;
    const float f0 = feat[((long long)b * CV + 0) * N3 + vox];
    const float f1 = feat[((long long)b * CV + 1) * N3 + vox];
#pragma unroll
    for (int o = 0; o < W; ++o)
      v0[((long long)b * W + o) * N3 + vox] =
          fmaf(Ps[o * CV + 1], f1, fmaf(Ps[o * CV], f0, Ps[W * CV + o]));
  }
}

// Tile loop shared by the gradient kernels: every block runs the same number
// of tiles; a thread without a voxel contributes zeros.
#define RPM_FNO_TILE_LOOP(total)                                                        \
  for (long long base = (long long)blockIdx.x * kThreads; base < (total);              \
       base += (long long)gridDim.x * kThreads)

// Gradient of the lift: gP = sum dv0 f^T, gp = sum dv0.
__global__ void __launch_bounds__(kThreads) k_lift_bwd(const float* __restrict__ dv0,
                                                       const float* __restrict__ feat,
                                                       float* __restrict__ part, long long N3,
                                                       int B) {
  using Acc = TileAcc<W, CV>;
  __shared__ float sL[W * Acc::LD];
  __shared__ float sR[CV * Acc::LD];
  Acc acc;
  acc.init();
  const long long total = N3 * B;
  const int t = threadIdx.x;
  RPM_FNO_TILE_LOOP(total) {
    const long long gidx = base + t;
    if (gidx < total) {
      const int b = (int)(gidx / N3);
      const long long vox = gidx - b * N3;
#pragma unroll
      for (int o = 0; o < W; ++o) sL[o * Acc::LD + t] = dv0[((long long)b * W + o) * N3 + vox];
#pragma unroll
      for (int c = 0; c < CV; ++c) sR[c * Acc::LD + t] = feat[((long long)b * CV + c) * N3 + vox];
    } else {
#pragma unroll
      for (int o = 0; o < W; ++o) sL[o * Acc::LD + t] = 0.f;
#pragma unroll
      for (int c = 0; c < CV; ++c) sR[c * Acc::LD + t] = 0.f;
    }
    __syncthreads();
    acc.step(sL, sR);
    __syncthreads();
  }
  acc.store(part + (long long)blockIdx.x * Acc::NE);
}

// Backward through layer l's pointwise part: dz = dv * gelu'(z) (dv on the last
// layer), dvprev = A^T dz, partials of gA = sum dz v^T and ga = sum dz.
__global__ void __launch_bounds__(kThreads) k_bwd_pw(const float* __restrict__ dv,
                                                     const float* __restrict__ zs,
                                                     const float* __restrict__ v,
                                                     const float* __restrict__ layer,
                                                     float* __restrict__ dz,
                                                     float* __restrict__ dvprev,
                                                     float* __restrict__ part, long long N3,
                                                     int B, int last) {
  using Acc = TileAcc4<W, W>;
  __shared__ __align__(16) float stage[Acc::SMEM];
  float* sL = stage;                     // [voxel][LDL]
  float* sR = stage + kThreads * Acc::LDL;
  __shared__ float As[W * W];
  for (int i = threadIdx.x; i < W * W; i += kThreads) As[i] = layer[i];
  __syncthreads();
  Acc acc;
  acc.init();
  const long long total = N3 * B;
  const int t = threadIdx.x;
  RPM_FNO_TILE_LOOP(total) {
    const long long gidx = base + t;
    float d[W], x[W];
    if (gidx < total) {
      const int b = (int)(gidx / N3);
      const long long vox = gidx - b * N3;
#pragma unroll
      for (int o = 0; o < W; ++o) {
        const long long at = ((long long)b * W + o) * N3 + vox;
        float g = dv[at];
        if (!last) g *= gelu_grad(zs[at]);
        d[o] = g;
        x[o] = v[at];
      }
#pragma unroll
      for (int o = 0; o < W; ++o) dz[((long long)b * W + o) * N3 + vox] = d[o];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < W; ++o) s = fmaf(As[o * W + c], d[o], s);
        dvprev[((long long)b * W + c) * N3 + vox] = s;
      }
    } else {
#pragma unroll
      for (int o = 0; o < W; ++o) d[o] = x[o] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      *reinterpret_cast<float4*>(sL + t * Acc::LDL + 4 * q) =
          make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
      *reinterpret_cast<float4*>(sR + t * Acc::LDR + 4 * q) =
          make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    }
    __syncthreads();
    acc.step(sL, sR);
    __syncthreads();
  }
  acc.store(part + (long long)blockIdx.x * Acc::NE, stage);
}

// Shared memory of k_head (floats): the two tiles, then per sample the
// contracted maps QE_b[o][c] (c < W) and qE_b[o] (c = W), then E.
size_t head_smem(int B) {
  return ((size_t)TileAcc4<NH, W>::SMEM + (size_t)B * COUT * (W + 1) + (size_t)B * CE) * 4;
}

// Localisation head: H = Q v + q (36 channels, channel 6 o + j = H[o][j]) and
// out[o] = sum_j H[o][j] E_bj, computed through the per-sample contracted map
// QE_b = sum_j Q[6 o + j] E_bj.  With a target: d = 2 (out - t) / nel,
// dH[o][j] = d[o] E_bj, dvL = Q^T dH = QE_b^T d, and partials of
// gQ = sum dH v^T, gq = sum dH and of sum (out - t)^2.
__global__ void __launch_bounds__(kThreads) k_head(const float* __restrict__ v,
                                                   const float* __restrict__ prm,
                                                   const float* __restrict__ Ed,
                                                   const float* __restrict__ target,
                                                   float* __restrict__ out,
                                                   float* __restrict__ dv,
                                                   float* __restrict__ part, long long N3, int B,
                                                   float inv_nel) {
  using Acc = TileAcc4<NH, W>;
  extern __shared__ float4 smem4[];
  float* sL = (float*)smem4;                 // [voxel][LDL]
  float* sR = sL + kThreads * Acc::LDL;      // [voxel][LDR]
  float* QE = (float*)smem4 + Acc::SMEM;     // [B][COUT][W + 1]
  float* Es = QE + B * COUT * (W + 1);       // [B][CE]
  __shared__ float red[kThreads / 32];
  for (int i = threadIdx.x; i < B * CE; i += kThreads) Es[i] = Ed[i];
  for (int i = threadIdx.x; i < B * COUT * (W + 1); i += kThreads) {
    const int b = i / (COUT * (W + 1)), r = i - b * (COUT * (W + 1));
    const int o = r / (W + 1), c = r - o * (W + 1);
    float s = 0.f;
    for (int j = 0; j < CE; ++j) {
      const float q = c < W ? prm[kOffQ + (o * CE + j) * W + c] : prm[kOffQ + NH * W + o * CE + j];
      s = fmaf(q, Ed[b * CE + j], s);
    }
    QE[i] = s;
  }
  __syncthreads();
  Acc acc;
  acc.init();
  float sq = 0.f;
  const long long total = N3 * B;
  const int t = threadIdx.x;
  RPM_FNO_TILE_LOOP(total) {
    const long long gidx = base + t;
    const bool have = gidx < total;
    if (have) {
      const int b = (int)(gidx / N3);
      const long long vox = gidx - b * N3;
      const float* qe = QE + b * COUT * (W + 1);
      float x[W];
#pragma unroll
      for (int c = 0; c < W; ++c) x[c] = v[((long long)b * W + c) * N3 + vox];
      float d[COUT];
#pragma unroll
      for (int o = 0; o < COUT; ++o) {
        float s = qe[o * (W + 1) + W];
#pragma unroll
        for (int c = 0; c < W; ++c) s = fmaf(qe[o * (W + 1) + c], x[c], s);
        const long long at = ((long long)b * COUT + o) * N3 + vox;
        if (out) out[at] = s;
        if (target) {
          const float diff = s - target[at];
          sq = fmaf(diff, diff, sq);
          d[o] = 2.f * diff * inv_nel;
        }
      }
      if (target) {
#pragma unroll
        for (int c = 0; c < W; ++c) {
          float s = 0.f;
#pragma unroll
          for (int o = 0; o < COUT; ++o) s = fmaf(qe[o * (W + 1) + c], d[o], s);
          dv[((long long)b * W + c) * N3 + vox] = s;
          sR[t * Acc::LDR + c] = x[c];
        }
#pragma unroll
        for (int o = 0; o < COUT; ++o)
#pragma unroll
          for (int j = 0; j < CE; ++j) sL[t * Acc::LDL + o * CE + j] = d[o] * Es[b * CE + j];
      }
    }
    if (target) {
      if (!have) {
#pragma unroll
        for (int k = 0; k < NH; ++k) sL[t * Acc::LDL + k] = 0.f;
#pragma unroll
        for (int c = 0; c < W; ++c) sR[t * Acc::LDR + c] = 0.f;
      }
      __syncthreads();
      acc.step(sL, sR);
      __syncthreads();
    }
  }
  if (!target) return;
  acc.store(part + (long long)blockIdx.x * kNeHead, (float*)smem4);   // after the loop's barrier
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((t & 31) == 0) red[t >> 5] = sq;
  __syncthreads();
  if (t == 0) {
    float s = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[(long long)blockIdx.x * kNeHead + kNeQ] = s;
  }
}

// dst[e] = sum over blocks of part[blk][e] (float64, fixed order) for e < n_grad;
// the entries after n_grad go to extra (float64).  A block takes 32
// consecutive entries (one per lane: coalesced rows); its 8 warps take every
// 8th partial row, then warp 0 adds the 8 warp sums in order.
constexpr int kRedWarps = 8;
__global__ void __launch_bounds__(32 * kRedWarps) k_reduce(const float* __restrict__ part,
                                                           int nblk, int stride, int n_grad,
                                                           int n_extra, float* __restrict__ dst,
                                                           double* __restrict__ extra) {
  __shared__ double sm[kRedWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  const int ne = n_grad + n_extra;
  double s = 0.0;
  if (e < ne) {
#pragma unroll 4
    for (int k = w; k < nblk; k += kRedWarps) s += (double)part[(long long)k * stride + e];
  }
  sm[w][lane] = s;
  __syncthreads();
  if (w == 0 && e < ne) {
    double t = 0.0;
    for (int q = 0; q < kRedWarps; ++q) t += sm[q][lane];
    if (e < n_grad)
      dst[e] = (float)t;
    else
      extra[e - n_grad] = t;
  }
}

int reduce_blocks(int ne) { return (ne + 31) / 32; }

// Adam with bias correction and decoupled weight decay.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long long n, float lr, float b1, float b2,
                       float eps, float wd, float bc1, float bc2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * ((a / bc1) / (sqrtf(b / bc2) + eps) + wd * p[i]);
  }
}

// Voxel features from a phase map: log10(Young / Young(phase 0)), Poisson ratio.
__global__ void k_features(const uint8_t* __restrict__ phase, const float2* __restrict__ tab,
                           long long n, float* __restrict__ feat) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 t = tab[phase[i]];
    feat[i] = t.x;
    feat[n + i] = t.y;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct rpm_fno {
  int N = 0, m = 0, L = 0, Bmax = 0, ncol = 0, YC = 8;
  bool tc = false;            // BF16 tensor-core transforms (precision RPM_FNO_BF16, N % 16 == 0)
  long long N3 = 0;
  size_t nparam = 0;
  cudaStream_t st = nullptr;
  float* params = nullptr;
  float* grads = nullptr;
  float* adam1 = nullptr;
  float* adam2 = nullptr;
  float* acts = nullptr;      // v_0..v_L, then z_0..z_{L-2}
  float* dvbuf = nullptr;     // two gradient buffers and dz
  float2* A2 = nullptr;
  float2* Bz = nullptr;
  float2* Vs = nullptr;       // per layer [ncol][Bmax][2m][W]
  float2* tw = nullptr;
  float* part = nullptr;
  double* extra = nullptr;
  float* Ed = nullptr;        // [Bmax][6]
  float* hE = nullptr;        // pinned staging of E
  double* hloss = nullptr;    // pinned
  float* feat1 = nullptr;     // warm start: features and output of one sample
  float* out1 = nullptr;
  float* eps0 = nullptr;      // rpm_fno_solve: the projected guess
  float2* ftab = nullptr;     // feature table per phase id (256)
  cudaEvent_t ev = nullptr;
  long long step = 0;
  size_t bytes = 0;
  std::string err;

  size_t act_floats() const { return (size_t)Bmax * W * N3; }
  float* v(int l) const { return acts + (size_t)l * act_floats(); }
  float* z(int l) const { return acts + (size_t)(L + 1 + l) * act_floats(); }
  float* dvb(int k) const { return dvbuf + (size_t)k * act_floats(); }
  float2* Vsl(int l) const { return Vs + (size_t)l * ncol * Bmax * 2 * m * W; }
  float* layer(int l) const { return params + layer_off(m, l); }
  float* glayer(int l) const { return grads + layer_off(m, l); }
};

namespace {

rpm_status ffail(rpm_fno* f, rpm_status s, const std::string& msg) {
  if (f) f->err = msg;
  return s;
}

bool fck(rpm_fno* f, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  f->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

int pw_blocks(long long total) {
  const long long t = (total + kThreads - 1) / kThreads;
  return (int)std::max(1LL, std::min<long long>(kPwBlocksMax, t));
}

cudaError_t set_smem(const void* k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

bool stage_E(rpm_fno* f, int B, const float* E_dir) {
  std::memcpy(f->hE, E_dir, sizeof(float) * CE * B);
  return fck(f, cudaMemcpyAsync(f->Ed, f->hE, sizeof(float) * CE * B, cudaMemcpyHostToDevice,
                                f->st),
             "E");
}

// Truncated forward xy transform of B samples into f->A2: the BF16
// tensor-core kernel when the network was created with RPM_FNO_BF16.
#define RPM_FNO_TC_SIZES(X) X(32) X(48) X(64) X(96) X(128)

void launch_xy_fwd(rpm_fno* f, const float* src, int B) {
  const int N = f->N, m = f->m;
  if (f->tc) {
    switch (N) {
#define RPM_CASE(NN)                                                                        \
  case NN:                                                                                  \
    k_xy_fwd_tc<NN><<<dim3(N, B), kThreads, xy_tc_smem(N, m), f->st>>>(src, f->A2, f->tw, m); \
    return;
      RPM_FNO_TC_SIZES(RPM_CASE)
#undef RPM_CASE
    }
  }
  k_xy_fwd<<<dim3(N, B), kThreads, xy_smem(N, m), f->st>>>(src, f->A2, f->tw, N, m);
}

// Forward spectral kernel of one layer: f->A2 -> f->Bz, V saved in Vs.
void launch_spec_fwd(rpm_fno* f, int B, const float2* R, float2* Vs) {
  const int N = f->N, m = f->m;
  if (f->tc) {
    switch (N) {
#define RPM_CASE(NN)                                                                           \
  case NN:                                                                                     \
    k_spec_fwd_tc<NN><<<f->ncol, kThreads, spec_tc_smem<NN>(m), f->st>>>(f->A2, R, Vs, f->Bz, \
                                                                         f->tw, m, B);         \
    return;
      RPM_FNO_TC_SIZES(RPM_CASE)
#undef RPM_CASE
    }
  }
  k_spec_fwd<<<dim3(f->ncol, B), kThreads, spec_smem(N, m), f->st>>>(f->A2, R, Vs, f->Bz, f->tw,
                                                                     N, m, B);
}

// Inverse xy transform of B samples from f->Bz (pointwise end as k_inv_xy).
template <bool BWD>
void launch_inv_xy(rpm_fno* f, int B, const float* layer, const float* vin, float* zsave,
                   float* vout, int last, float inv_n3) {
  const int N = f->N, m = f->m;
  const dim3 grid(N / f->YC, N, B);
  if (f->tc) {
    switch (N) {
#define RPM_CASE(NN)                                                                     \
  case NN:                                                                               \
    k_inv_xy_tc<BWD, NN><<<grid, kThreads, inv_tc_smem(N, m, f->YC), f->st>>>(          \
        f->Bz, f->tw, layer, vin, zsave, vout, m, f->YC, last, inv_n3);                 \
    return;
      RPM_FNO_TC_SIZES(RPM_CASE)
#undef RPM_CASE
    }
  }
  k_inv_xy<BWD><<<grid, kThreads, inv_smem(m, f->YC), f->st>>>(f->Bz, f->tw, layer, vin, zsave,
                                                              vout, N, m, f->YC, last, inv_n3);
}

// Forward pass; keeps v_l and z_l.  out (optional), target (optional: then the
// head also writes dv_L into dvb(0) and its partials).
bool run_forward(rpm_fno* f, int B, const float* feat, const float* target, float* out) {
  const int N = f->N, m = f->m, L = f->L;
  const long long total = f->N3 * B;
  const int nb = pw_blocks(total);
  const float inv_n3 = 1.f / (float)f->N3;
  k_lift<<<nb, kThreads, 0, f->st>>>(feat, f->params, f->v(0), f->N3, B);
  if (!fck(f, cudaGetLastError(), "lift")) return false;
  for (int l = 0; l < L; ++l) {
    launch_xy_fwd(f, f->v(l), B);
    launch_spec_fwd(f, B, (const float2*)(f->layer(l) + kLayerHead), f->Vsl(l));
    const int last = (l == L - 1);
    launch_inv_xy<false>(f, B, f->layer(l), f->v(l), last ? nullptr : f->z(l), f->v(l + 1), last,
                         inv_n3);
    if (!fck(f, cudaGetLastError(), "layer")) return false;
  }
  const float inv_nel = 1.f / (float)(total * COUT);
  k_head<<<nb, kThreads, head_smem(B), f->st>>>(f->v(L), f->params, f->Ed, target, out,
                                                 f->dvb(0), f->part, f->N3, B, inv_nel);
  if (!fck(f, cudaGetLastError(), "head")) return false;
  if (target) {
    k_reduce<<<reduce_blocks(kNeHead), 32 * kRedWarps, 0, f->st>>>(f->part, nb, kNeHead, kNeQ, 1,
                                                                   f->grads + kOffQ, f->extra);
    if (!fck(f, cudaGetLastError(), "reduce head")) return false;
  }
  return true;
}

bool run_backward(rpm_fno* f, int B, const float* feat) {
  const int N = f->N, m = f->m, L = f->L;
  const long long total = f->N3 * B;
  const int nb = pw_blocks(total);
  const float inv_n3 = 1.f / (float)f->N3;
  int cur = 0;   // dvb(cur) holds dL/dv_{l+1}
  for (int l = L - 1; l >= 0; --l) {
    const int last = (l == L - 1);
    float* dz = f->dvb(2);
    float* prev = f->dvb(1 - cur);
    k_bwd_pw<<<nb, kThreads, 0, f->st>>>(f->dvb(cur), last ? nullptr : f->z(l), f->v(l),
                                         f->layer(l), dz, prev, f->part, f->N3, B, last);
    k_reduce<<<reduce_blocks(kNeA), 32 * kRedWarps, 0, f->st>>>(f->part, nb, kNeA, kNeA, 0,
                                                                f->glayer(l), nullptr);
    launch_xy_fwd(f, dz, B);
    k_spec_bwd<<<f->ncol, kThreads, spec_smem(N, m), f->st>>>(
        f->A2, (const float2*)(f->layer(l) + kLayerHead), f->Vsl(l),
        (float2*)(f->glayer(l) + kLayerHead), f->Bz, f->tw, N, m, B, inv_n3);
    launch_inv_xy<true>(f, B, nullptr, nullptr, nullptr, prev, 0, inv_n3);
    if (!fck(f, cudaGetLastError(), "layer backward")) return false;
    cur = 1 - cur;
  }
  k_lift_bwd<<<nb, kThreads, 0, f->st>>>(f->dvb(cur), feat, f->part, f->N3, B);
  k_reduce<<<reduce_blocks(kNeP), 32 * kRedWarps, 0, f->st>>>(f->part, nb, kNeP, kNeP, 0,
                                                               f->grads + kOffP, nullptr);
  return fck(f, cudaGetLastError(), "lift backward");
}

// Shared-memory limits of the tensor-core kernels (per grid side: sixteen
// rows per k_inv_xy block up to N = 64, eight above; any number of modes).
bool set_tc_smem() {
#define RPM_CASE(NN)                                                                         \
  if (set_smem((const void*)k_xy_fwd_tc<NN>, xy_tc_smem(NN, kMaxModes)) != cudaSuccess ||    \
      set_smem((const void*)k_inv_xy_tc<false, NN>,                                         \
               inv_tc_smem(NN, kMaxModes, NN <= 64 ? 16 : 8)) != cudaSuccess ||             \
      set_smem((const void*)k_inv_xy_tc<true, NN>,                                          \
               inv_tc_smem(NN, kMaxModes, NN <= 64 ? 16 : 8)) != cudaSuccess ||             \
      set_smem((const void*)k_spec_fwd_tc<NN>, spec_tc_smem<NN>(kMaxModes)) != cudaSuccess)   \
    return false;
  RPM_FNO_TC_SIZES(RPM_CASE)
#undef RPM_CASE
  return true;
}

bool valid_batch(rpm_fno* f, int B) { return f && B >= 1 && B <= f->Bmax; }

}  // namespace

extern "C" {

size_t rpm_fno_param_count(int modes, int layers) {
  if (modes < 1 || modes > kMaxModes || layers < 1 || layers > RPM_FNO_MAX_LAYERS) return 0;
  return layer_off(modes, layers);
}

rpm_status rpm_fno_create(const rpm_fno_config* cfg, void* cuda_stream, rpm_fno** out) {
  if (!cfg || !out) return RPM_ERR_INVALID_ARG;
  *out = nullptr;
  const int N = cfg->n, m = cfg->modes, L = cfg->layers, B = cfg->max_batch;
  if (cfg->precision != RPM_FNO_FP32 && cfg->precision != RPM_FNO_BF16) return RPM_ERR_INVALID_ARG;
  if (m < 1 || m > kMaxModes || L < 1 || L > RPM_FNO_MAX_LAYERS || B < 1 ||
      B > RPM_FNO_MAX_BATCH || N < 24 ||
      N > RPM_FNO_MAX_N || N % 8 != 0 || N < 2 * m)
    return RPM_ERR_INVALID_ARG;
  rpm_fno* f = new rpm_fno();
  f->N = N;
  f->m = m;
  f->L = L;
  f->Bmax = B;
  f->ncol = 2 * m * m;
  f->N3 = (long long)N * N * N;
  f->nparam = rpm_fno_param_count(m, L);
  f->st = (cudaStream_t)cuda_stream;
  f->YC = (N <= 64 && N % 16 == 0) ? 16 : 8;   // rows per k_inv_xy block (divides N)
  f->tc = cfg->precision == RPM_FNO_BF16 && N % 16 == 0;
  auto alloc = [&](void** p, size_t b) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(b, 256));
    if (e == cudaSuccess) f->bytes += b;
    return e == cudaSuccess;
  };
  const size_t P = f->nparam * sizeof(float);
  const size_t act = f->act_floats() * sizeof(float);
  const size_t colb = (size_t)B * N * f->ncol * W * sizeof(float2);
  const size_t vsb = (size_t)L * f->ncol * B * 2 * m * W * sizeof(float2);
  const size_t partb = (size_t)kPwBlocksMax * kNeA * sizeof(float);   // largest row
  const bool ok =
      alloc((void**)&f->params, P) && alloc((void**)&f->grads, P) &&
      alloc((void**)&f->adam1, P) && alloc((void**)&f->adam2, P) &&
      alloc((void**)&f->acts, act * (2 * L)) && alloc((void**)&f->dvbuf, act * 3) &&
      alloc((void**)&f->A2, colb) && alloc((void**)&f->Bz, colb) && alloc((void**)&f->Vs, vsb) &&
      alloc((void**)&f->tw, N * sizeof(float2)) && alloc((void**)&f->part, partb) &&
      alloc((void**)&f->extra, 64) && alloc((void**)&f->Ed, B * CE * sizeof(float)) &&
      alloc((void**)&f->feat1, f->N3 * CV * sizeof(float)) &&
      alloc((void**)&f->out1, f->N3 * COUT * sizeof(float)) &&
      alloc((void**)&f->eps0, f->N3 * COUT * sizeof(float)) &&
      alloc((void**)&f->ftab, 256 * sizeof(float2));
  if (!ok || cudaMallocHost((void**)&f->hE, B * CE * sizeof(float)) != cudaSuccess ||
      cudaMallocHost((void**)&f->hloss, 64) != cudaSuccess ||
      cudaEventCreateWithFlags(&f->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rpm_fno_destroy(f);
    return RPM_ERR_OOM;
  }
  std::vector<float2> tw(N);
  for (int j = 0; j < N; ++j) {
    const double a = -2.0 * M_PI * (double)j / (double)N;
    tw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  const size_t smax = std::max(std::max(xy_smem(N, m), xy_tc_smem(N, m)),
                               std::max(spec_smem(N, m), std::max(inv_smem(m, f->YC),
                                                                  inv_tc_smem(N, m, f->YC))));

  if (smax > 227 * 1024 ||
      cudaMemcpyAsync(f->tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, f->st) !=
          cudaSuccess ||
      cudaMemsetAsync(f->params, 0, P, f->st) != cudaSuccess ||
      cudaMemsetAsync(f->grads, 0, P, f->st) != cudaSuccess ||
      cudaMemsetAsync(f->adam1, 0, P, f->st) != cudaSuccess ||
      cudaMemsetAsync(f->adam2, 0, P, f->st) != cudaSuccess ||
      // the attribute is per kernel, not per network: allow the largest configuration
      set_smem((const void*)k_xy_fwd, xy_smem(RPM_FNO_MAX_N, kMaxModes)) != cudaSuccess ||
      !set_tc_smem() ||
      set_smem((const void*)k_spec_fwd, spec_smem(RPM_FNO_MAX_N, kMaxModes)) != cudaSuccess ||
      set_smem((const void*)k_spec_bwd, spec_smem(RPM_FNO_MAX_N, kMaxModes)) != cudaSuccess ||
      set_smem((const void*)k_inv_xy<false>, inv_smem(kMaxModes, 16)) != cudaSuccess ||
      set_smem((const void*)k_inv_xy<true>, inv_smem(kMaxModes, 16)) != cudaSuccess ||

      set_smem((const void*)k_head, head_smem(RPM_FNO_MAX_BATCH)) != cudaSuccess ||
      cudaStreamSynchronize(f->st) != cudaSuccess) {
    cudaGetLastError();
    rpm_fno_destroy(f);
    return RPM_ERR_CUDA;
  }
  *out = f;
  return RPM_OK;
}

rpm_status rpm_fno_set_params(rpm_fno* f, const float* params) {
  if (!f || !params) return ffail(f, RPM_ERR_INVALID_ARG, "null argument");
  const size_t P = f->nparam * sizeof(float);
  if (!fck(f, cudaMemcpyAsync(f->params, params, P, cudaMemcpyHostToDevice, f->st), "params") ||
      !fck(f, cudaMemsetAsync(f->adam1, 0, P, f->st), "adam") ||
      !fck(f, cudaMemsetAsync(f->adam2, 0, P, f->st), "adam") ||
      !fck(f, cudaStreamSynchronize(f->st), "sync"))
    return RPM_ERR_CUDA;
  f->step = 0;
  return RPM_OK;
}

static rpm_status copy_out(rpm_fno* f, const float* src, float* dst) {
  if (!f || !dst) return ffail(f, RPM_ERR_INVALID_ARG, "null argument");
  if (!fck(f, cudaMemcpyAsync(dst, src, f->nparam * sizeof(float), cudaMemcpyDeviceToHost, f->st),
           "copy") ||
      !fck(f, cudaStreamSynchronize(f->st), "sync"))
    return RPM_ERR_CUDA;
  return RPM_OK;
}

rpm_status rpm_fno_get_params(rpm_fno* f, float* params) {
  return copy_out(f, f ? f->params : nullptr, params);
}

rpm_status rpm_fno_get_grads(rpm_fno* f, float* grads) {
  return copy_out(f, f ? f->grads : nullptr, grads);
}

rpm_status rpm_fno_forward(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                           float* out) {
  if (!valid_batch(f, batch) || !feat || !E_dir || !out)
    return ffail(f, RPM_ERR_INVALID_ARG, "bad forward arguments");
  if (!stage_E(f, batch, E_dir) || !run_forward(f, batch, feat, nullptr, out))
    return RPM_ERR_CUDA;
  return RPM_OK;
}

rpm_status rpm_fno_loss_grad(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                             const float* target, double* loss) {
  if (!valid_batch(f, batch) || !feat || !E_dir || !target)
    return ffail(f, RPM_ERR_INVALID_ARG, "bad loss_grad arguments");
  if (!stage_E(f, batch, E_dir) || !run_forward(f, batch, feat, target, nullptr) ||
      !run_backward(f, batch, feat))
    return RPM_ERR_CUDA;
  if (loss) {
    if (!fck(f, cudaMemcpyAsync(f->hloss, f->extra, 8, cudaMemcpyDeviceToHost, f->st), "loss") ||
        !fck(f, cudaStreamSynchronize(f->st), "sync"))
      return RPM_ERR_CUDA;
    *loss = f->hloss[0] / ((double)f->N3 * batch * COUT);
  }
  return RPM_OK;
}

rpm_status rpm_fno_adam_step(rpm_fno* f, const rpm_fno_adam* o) {
  if (!f || !o || !(o->lr >= 0) || !(o->beta1 >= 0 && o->beta1 < 1) ||
      !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0) || !(o->weight_decay >= 0))
    return ffail(f, RPM_ERR_INVALID_ARG, "bad Adam options");
  ++f->step;
  const float bc1 = (float)(1.0 - std::pow((double)o->beta1, (double)f->step));
  const float bc2 = (float)(1.0 - std::pow((double)o->beta2, (double)f->step));
  k_adam<<<4 * 152, 256, 0, f->st>>>(f->params, f->grads, f->adam1, f->adam2,
                                     (long long)f->nparam, o->lr, o->beta1, o->beta2, o->eps,
                                     o->weight_decay, bc1, bc2);
  return fck(f, cudaGetLastError(), "adam") ? RPM_OK : RPM_ERR_CUDA;
}

rpm_status rpm_fno_train_step(rpm_fno* f, int batch, const float* feat, const float* E_dir,
                              const float* target, const rpm_fno_adam* opt, double* loss) {
  if (!opt) return ffail(f, RPM_ERR_INVALID_ARG, "null Adam options");
  rpm_status s = rpm_fno_loss_grad(f, batch, feat, E_dir, target, loss);
  if (s != RPM_OK) return s;
  return rpm_fno_adam_step(f, opt);
}

static rpm_status features_on(const uint8_t* phase, long long n, int n_phases,
                              const rpm_iso* phases, float* feat, float2* tab_dev,
                              cudaStream_t st) {
  std::vector<float2> tab(256, make_float2(0.f, 0.f));
  const double l0 = phases[0].lambda, m0 = phases[0].mu;
  const double y0 = m0 * (3 * l0 + 2 * m0) / (l0 + m0);
  for (int i = 0; i < n_phases; ++i) {
    const double l = phases[i].lambda, m = phases[i].mu;
    const double y = m * (3 * l + 2 * m) / (l + m);
    tab[i] = make_float2((float)std::log10(y / y0), (float)(l / (2 * (l + m))));
  }
  if (cudaMemcpyAsync(tab_dev, tab.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return RPM_ERR_CUDA;
  k_features<<<4 * 152, 256, 0, st>>>(phase, tab_dev, n, feat);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return RPM_ERR_CUDA;
  return RPM_OK;
}

static bool valid_moduli(int n_phases, const rpm_iso* phases) {
  if (n_phases < 1 || n_phases > 256 || !phases) return false;
  for (int i = 0; i < n_phases; ++i)
    if (!(phases[i].mu > 0) || !(phases[i].lambda + phases[i].mu > 0)) return false;
  return true;
}

rpm_status rpm_fno_features(const uint8_t* phase, long long n, int n_phases,
                            const rpm_iso* phases, float* feat, void* cuda_stream) {
  if (!phase || !feat || n < 1 || !valid_moduli(n_phases, phases)) return RPM_ERR_INVALID_ARG;
  float2* tab = nullptr;
  if (cudaMalloc((void**)&tab, 256 * sizeof(float2)) != cudaSuccess) return RPM_ERR_OOM;
  const rpm_status s =
      features_on(phase, n, n_phases, phases, feat, tab, (cudaStream_t)cuda_stream);
  cudaFree(tab);
  return s;
}

rpm_status rpm_fno_warm_start(rpm_fno* f, rpm_ctx* ctx, const double E[6], float* eps0) {
  if (!f || !ctx || !E || !eps0) return ffail(f, RPM_ERR_INVALID_ARG, "null argument");
  rpm::CellView cv{};
  if (!rpm::ctx_cell_view(ctx, &cv)) return ffail(f, RPM_ERR_INVALID_ARG, "bad context");
  if (cv.nx != f->N || cv.ny != f->N || cv.nz != f->N)
    return ffail(f, RPM_ERR_INVALID_ARG, "context grid differs from the network grid");
  if (!valid_moduli(cv.n_phases, cv.phases)) return ffail(f, RPM_ERR_INVALID_ARG, "bad moduli");
  double nrm = 0;
  for (int k = 0; k < 6; ++k) nrm += (k < 3 ? 1.0 : 2.0) * E[k] * E[k];
  nrm = std::sqrt(nrm);
  if (!(nrm > 0) || !std::isfinite(nrm)) return ffail(f, RPM_ERR_INVALID_ARG, "E must be nonzero");
  // the phase map is written on the context stream: order the network after it
  if (!fck(f, cudaEventRecord(f->ev, cv.st), "event") ||
      !fck(f, cudaStreamWaitEvent(f->st, f->ev, 0), "event"))
    return RPM_ERR_CUDA;
  if (features_on(cv.phase, f->N3, cv.n_phases, cv.phases, f->feat1, f->ftab, f->st) != RPM_OK)
    return ffail(f, RPM_ERR_CUDA, "features");
  float e[6];
  for (int k = 0; k < 6; ++k) e[k] = (float)E[k];   // the output is linear in E
  if (!stage_E(f, 1, e) || !run_forward(f, 1, f->feat1, nullptr, f->out1) ||
      !fck(f, cudaStreamSynchronize(f->st), "sync"))
    return RPM_ERR_CUDA;
  const rpm_status s = rpm_apply_gamma(ctx, f->out1, E, eps0, RPM_GAMMA_PROJECT);
  if (s != RPM_OK) return ffail(f, s, std::string("projection: ") + rpm_last_error(ctx));
  if (!fck(f, cudaStreamSynchronize(cv.st), "sync")) return RPM_ERR_CUDA;
  return RPM_OK;
}

rpm_status rpm_fno_solve(rpm_fno* f, rpm_ctx* ctx, const double E[6], float* eps_out,
                         float* sig_out, int out_on_host, rpm_solve_info* info, int* used_guess) {
  if (used_guess) *used_guess = 0;
  rpm_status s = rpm_fno_warm_start(f, ctx, E, f ? f->eps0 : nullptr);
  if (s != RPM_OK) return s;
  rpm_solve_info first{};
  s = rpm_solve(ctx, E, f->eps0, eps_out, sig_out, out_on_host, &first);
  if (s == RPM_OK) {
    if (used_guess) *used_guess = 1;
    if (info) *info = first;
    return RPM_OK;
  }
  if (s != RPM_ERR_DIVERGED && s != RPM_ERR_NOT_CONVERGED) {
    if (info) *info = first;
    return s;
  }
  // the cold start is the fallback: the context's own form from eps0 = E
  rpm_solve_info second{};
  s = rpm_solve(ctx, E, nullptr, eps_out, sig_out, out_on_host, &second);
  second.gamma_applies += first.gamma_applies;
  second.ms += first.ms;
  second.launches += first.launches;
  if (info) *info = second;
  return s;
}

size_t rpm_fno_device_bytes(const rpm_fno* f) { return f ? f->bytes : 0; }

const char* rpm_fno_last_error(const rpm_fno* f) { return f ? f->err.c_str() : "null network"; }

void rpm_fno_destroy(rpm_fno* f) {
  if (!f) return;
  void* dev[] = {f->params, f->grads, f->adam1, f->adam2, f->acts, f->dvbuf,
                 f->A2,     f->Bz,    f->Vs,    f->tw,    f->part, f->extra,
                 f->Ed,     f->feat1, f->out1,  f->eps0,  f->ftab};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (f->hE) cudaFreeHost(f->hE);
  if (f->hloss) cudaFreeHost(f->hloss);
  if (f->ev) cudaEventDestroy(f->ev);
  delete f;
}

}  // extern "C"
