// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rpm.h"

namespace rpm {

constexpr int kMaxBasis = 256;   // largest unstable basis (projections run in chunks of 32)

// How the zero frequency and the input are treated by one Gamma0 application.
enum GammaMode {
  GM_FULL_MAP = 0,   // input eps; output F(eps) = E - Gamma0 * ((C - C0) : eps)
  GM_LINEAR = 1,     // input eps; output F_u eps = -Gamma0 * ((C - C0) : eps)
  GM_RAW_TAU = 2,    // input tau; output -Gamma0 * tau (zero mean)
};

// Device-side description of one grid, its FFT tables and the materials.
struct GridDev {
  int nx, ny, nz;        // each 2^a 3^b
  int nxh;               // nx / 2
  long long n;           // voxels
  int plane;             // ny * (nxh + 1): half-spectrum slots per z-plane
  // tables (device pointers into one allocation)
  const float2* tw_x;    // W_{nxh}^(n2*k1), nxh entries
  const float2* tw_y;    // W_{ny}^(n2*k1), ny entries
  const float2* tw_z;    // W_{nz}^(n2*k1), nz entries
  const float2* r2c_w;   // W_{nx}^k, k = 0..nxh
  const int2* fx;        // per x slot: (signed frequency m, nyquist flag)
  const int2* fy;        // per y slot
  const uint8_t* phase;  // [nz][ny][nx]
  const float2* dmat;    // per phase: (lam - lam0, mu - mu0)
  const float2* cmat;    // per phase: (lam, mu)
  int n_phases;
  float lam0, mu0;
  float inv_lx, inv_ly, inv_lz;   // 1 / L_j (frequency scaling)
  int nyquist;           // 0: zero mixed Nyquist frequencies, 1: signed
  int plane_v;           // x/y passes: 0 fused where available, 1 whole-plane, 2 five-pass
  int pencil_t;          // z pass: 0 fused where available, else the default tile;
                         // 1 half, 2 twice the default pencils; 3 the default tile
  int* err;              // device flag set to 1 when a bounded wait of a kernel gave up
};

// One Gamma0 application: in [6][n] -> out [6][n] through the spectrum
// scratch spec [6][nz][plane] (float2).  E (6 tensor components) is only
// used in GM_FULL_MAP.  A non-null `add` [6][n] is added to the output (in
// the last pass where the fused kernels run, else by one more launch).
// Returns a CUDA error code.
cudaError_t launch_apply_gamma(const GridDev& g, const float* in, float* out, float2* spec,
                               const double E[6], int mode, cudaStream_t st,
                               const float* add = nullptr);
int gamma_add_launches(const GridDev& g, const float* out, const float* add, const float2* spec);

// Algorithm 3 as one map application: eps_b = the Gamma0 map of `in` under g
// (whose material table holds s_b's moduli, E = Eb), then the post-step
// out = (C + C0)^-1 : (s_a(in) + C0 : eps_b) with the per-phase table `post`
// (see launch_polarization_post).  On the fused plane passes the post-step
// is the last pass's epilogue and eb is not touched; otherwise eb is the
// scratch of a separate post-step launch.
cudaError_t launch_polarization_map(const GridDev& g, const float4* post, const float* in,
                                    float* eb, float* out, float2* spec, const double Eb[6],
                                    int mode, cudaStream_t st);
int polarization_launches(const GridDev& g, const float* in, const float* out,
                          const float2* spec);

// One block whose asynchronous-copy barrier wait can never complete:
// out[0] = 1 once the bounded wait has given up by itself.
cudaError_t launch_wait_selfcheck(int* out, cudaStream_t st);

bool grid_supported(int nx, int ny, int nz);
int gamma_launches(const GridDev& g);  // kernels per Gamma0 application (3 or 5)
int pencil_tile(const GridDev& g);     // pencils per pass-B block for g.pencil_t
int plane_variant(const GridDev& g);   // plane kernels g.plane_v resolves to (0, 1, 2)
bool fused_z_pass(const GridDev& g);   // g.pencil_t resolves to the fused z kernel

// ---- field kernels (field_kernels.cu) -------------------------------------
// Partial sums per block, then one finishing block; see the definitions.
int dots_blocks_for(long long n);
int dots_launches(int K);
int combine_launches(int K);
int stress_blocks_for(long long n);
cudaError_t launch_dots(const float* x, const float* x_minus /*nullable*/, const float* Y,
                        long long ystride, int K, long long n, double* partials, int nblk,
                        cudaStream_t st);
cudaError_t launch_reduce_partials(const double* partials, int nblk, int m, double* out,
                                   cudaStream_t st);
// launch_dots + launch_reduce_partials (+ launch_newton when M is given, p = K)
// in one launch, for K <= 32; ticket: a device counter that is zero on entry.
cudaError_t launch_dots_fused(const float* x, const float* x_minus, const float* Y,
                              long long ystride, int K, long long n, double* partials, int nblk,
                              double* sums, unsigned int* ticket, const double* M, double* c,
                              double* res_out, double inv_norm, cudaStream_t st);
cudaError_t launch_combine(float* out, const float* x, float xscale, const float* Y,
                           long long ystride, int K, const double* coef, float cscale,
                           long long n, cudaStream_t st);
cudaError_t launch_axpby(float* out, float a, const float* x, float b, const float* y, long long n,
                         cudaStream_t st);
cudaError_t launch_stress(const GridDev& g, const float* eps, float* sig /*nullable*/,
                          double* partials, int nblk, cudaStream_t st);
cudaError_t launch_fill(float* f, const double E[6], long long n, cudaStream_t st);
// Algorithm 3's last step: out = (C + C0)^-1 : (s_a(eps) + C0 : eps_b), with per-phase
// table post[r] = (lam_a, mu_a, k_s, h_s); s_a = lam_a tr(eps) I + 2 mu_a eps and
// (C + C0) = (lam_s, mu_s), k_s = lam_s / (3 lam_s + 2 mu_s), h_s = 1 / (2 mu_s).
cudaError_t launch_polarization_post(const GridDev& g, const float4* post, const float* eps,
                                     const float* eps_b, float* out, cudaStream_t st);
cudaError_t launch_newton(const double* sums, int p, const double* M, double* c, double* res_out,
                          double inv_norm, cudaStream_t st);

// ---- context view for the learned warm start (rpm_api.cu) ----------------
struct CellView {
  int nx, ny, nz;
  const uint8_t* phase;   // device [nz][ny][nx]
  const rpm_iso* phases;  // host, n_phases entries
  int n_phases;
  cudaStream_t st;        // the context stream
};
bool ctx_cell_view(const rpm_ctx* c, CellView* v);

}  // namespace rpm
