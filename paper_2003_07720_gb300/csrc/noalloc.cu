// rpm_apply_gamma_noalloc: the Gamma0 application of rpm_apply_gamma for
// callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application that owns
// every byte of device memory through its own pool or plug-in allocator, or a
// latency-critical loop where cudaMalloc's implicit device synchronisation is
// not acceptable.  This entry point needs no context and allocates nothing.
// Its scratch -- the half spectrum and the FFT, frequency and material tables
// -- lives in file-scope __device__ arrays of fixed size, which every GPU that
// loads the library keeps until the process exits.  The caller passes the
// phase map, the input field and the output field.
#include <cmath>
#include <cstring>

#include "fft_smem.cuh"
#include "rpm.h"
#include "rpm_internal.h"

namespace rpm {
namespace {

// Largest grid served: nx = ny <= 64, nz <= 64 (spectrum 6 * 64 * 64 * 33
// complex values = 6.5 MB).
constexpr int kNaMax = 64;
constexpr size_t kNaSpec = (size_t)6 * kNaMax * kNaMax * (kNaMax / 2 + 1);

static __device__ __align__(256) float2 g_na_spec[kNaSpec];
static __device__ __align__(256) float2 g_na_tw[3 * kNaMax];        // x (nx/2), y, z twiddles
static __device__ __align__(256) float2 g_na_r2c[kNaMax / 2 + 1];
static __device__ __align__(256) int2 g_na_f[kNaMax / 2 + 1 + kNaMax];  // x slots, then y slots
static __device__ __align__(256) float2 g_na_mat[2 * 256];           // (dlam, dmu), (lam, mu)

struct NaAddr {
  bool ready = false;
  float2* spec = nullptr;
  float2* tw = nullptr;
  float2* r2c = nullptr;
  int2* f = nullptr;
  float2* mat = nullptr;
};
constexpr int kNaDevices = 64;
static NaAddr g_na_addr[kNaDevices];   // host-side: device addresses per device ordinal

// Device addresses of the arrays on the current device (host code may not use
// the array names as pointers); looked up once per device.
cudaError_t na_setup(int dev, NaAddr** out) {
  NaAddr& a = g_na_addr[dev];
  if (!a.ready) {
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void**)&a.spec, g_na_spec)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.tw, g_na_tw)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.r2c, g_na_r2c)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.f, g_na_f)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&a.mat, g_na_mat)) != cudaSuccess) return e;
    a.ready = true;
  }
  *out = &a;
  return cudaSuccess;
}

void na_twiddles(int L, float2* out) {
  const int N1 = split_n1(L), N2 = split_n2(L);
  for (int n2 = 0; n2 < N2; ++n2)
    for (int k1 = 0; k1 < N1; ++k1) {
      const double a = -2.0 * M_PI * (double)n2 * (double)k1 / (double)L;
      out[n2 * N1 + k1] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
}

}  // namespace
}  // namespace rpm

using namespace rpm;

extern "C" rpm_status rpm_apply_gamma_noalloc(const rpm_grid* grid, const uint8_t* phase,
                                              int n_phases, const rpm_iso* phases, rpm_iso c0,
                                              const float* in, const double E[6], float* out,
                                              int flags, void* cuda_stream) {
  if (!grid || !phase || !phases || !in || !out || n_phases < 1 || n_phases > 256)
    return RPM_ERR_INVALID_ARG;
  if (flags < RPM_GAMMA_FULL_MAP || flags > RPM_GAMMA_RAW_TAU) return RPM_ERR_INVALID_ARG;
  if (flags == RPM_GAMMA_FULL_MAP && !E) return RPM_ERR_INVALID_ARG;
  if (in == out) return RPM_ERR_INVALID_ARG;
  if (!(c0.mu > 0) || !(c0.lambda + 2 * c0.mu > 0)) return RPM_ERR_INVALID_ARG;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (!grid_supported(nx, ny, nz)) return RPM_ERR_UNSUPPORTED_GRID;
  if (nx > kNaMax || ny > kNaMax || nz > kNaMax) return RPM_ERR_UNSUPPORTED_GRID;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaDevices) return RPM_ERR_CUDA;
  NaAddr* a = nullptr;
  if (na_setup(dev, &a) != cudaSuccess) return RPM_ERR_CUDA;

  // host tables (the same definitions as a context's), then stream-ordered
  // copies into the file-scope arrays
  const int nxh = nx / 2;
  float2 tw[3 * kNaMax];
  na_twiddles(nxh, tw);
  na_twiddles(ny, tw + kNaMax);
  na_twiddles(nz, tw + 2 * kNaMax);
  float2 r2c[kNaMax / 2 + 1];
  for (int k = 0; k <= nxh; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)nx;
    r2c[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  int2 f[kNaMax / 2 + 1 + kNaMax];
  for (int s = 0; s <= nxh; ++s) {
    const int k = s < nxh ? freq_of_rt(nxh, s) : nxh;
    const bool nyq = (k == nxh);
    f[s] = make_int2(nyq ? -k : k, nyq ? 1 : 0);
  }
  for (int s = 0; s < ny; ++s) {
    const int k = freq_of_rt(ny, s);
    f[nxh + 1 + s] = make_int2((2 * k < ny) ? k : k - ny, (ny % 2 == 0 && 2 * k == ny) ? 1 : 0);
  }
  float2 mat[2 * 256];
  std::memset(mat, 0, sizeof(mat));
  for (int i = 0; i < n_phases; ++i) {
    mat[i] = make_float2((float)(phases[i].lambda - c0.lambda), (float)(phases[i].mu - c0.mu));
    mat[256 + i] = make_float2((float)phases[i].lambda, (float)phases[i].mu);
  }
  if (cudaMemcpyAsync(a->tw, tw, sizeof(tw), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(a->r2c, r2c, sizeof(r2c), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(a->f, f, sizeof(f), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(a->mat, mat, sizeof(mat), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RPM_ERR_CUDA;
  // the host arrays above live on this stack frame: wait for the copies
  if (cudaStreamSynchronize(st) != cudaSuccess) return RPM_ERR_CUDA;

  GridDev g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxh = nxh;
  g.n = (long long)nx * ny * nz;
  g.plane = ny * (nxh + 1);
  g.tw_x = a->tw;
  g.tw_y = a->tw + kNaMax;
  g.tw_z = a->tw + 2 * kNaMax;
  g.r2c_w = a->r2c;
  g.fx = a->f;
  g.fy = a->f + nxh + 1;
  g.phase = phase;
  g.dmat = a->mat;
  g.cmat = a->mat + 256;
  g.n_phases = n_phases;
  g.lam0 = (float)c0.lambda;
  g.mu0 = (float)c0.mu;
  g.inv_lx = (float)(1.0 / (grid->lx > 0 ? grid->lx : 1.0));
  g.inv_ly = (float)(1.0 / (grid->ly > 0 ? grid->ly : 1.0));
  g.inv_lz = (float)(1.0 / (grid->lz > 0 ? grid->lz : 1.0));
  g.nyquist = RPM_NYQ_ZERO_MIXED;
  // the spectrum is fully written by the first pass before it is read: no clearing
  if (launch_apply_gamma(g, in, out, a->spec, E, flags, st) != cudaSuccess) return RPM_ERR_CUDA;
  return RPM_OK;
}
