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
#include <mutex>

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
static __device__ __align__(256) int g_na_err[4];                    // bounded-wait flag

// Per device: the arrays' device addresses and a host copy of the tables
// last uploaded there, so that repeated calls with the same grid, materials
// and C0 upload nothing.
struct NaDevice {
  std::once_flag once;
  cudaError_t setup = cudaSuccess;
  float2* spec = nullptr;
  float2* tw = nullptr;
  float2* r2c = nullptr;
  int2* f = nullptr;
  float2* mat = nullptr;
  int* err = nullptr;
  std::mutex mu;            // guards the key below
  bool have_key = false;
  int key_grid[3] = {0, 0, 0};
  float2 key_mat[2 * 256];
};
constexpr int kNaDevices = 64;
static NaDevice g_na_dev[kNaDevices];

// Device addresses of the arrays on the current device: host code may not
// use the array names as pointers.  Looked up once per device (std::call_once,
// so concurrent first calls from several host threads are safe).
cudaError_t na_setup(int dev, NaDevice** out) {
  NaDevice& d = g_na_dev[dev];
  std::call_once(d.once, [&d]() {
    cudaError_t e;
    if ((e = cudaGetSymbolAddress((void**)&d.spec, g_na_spec)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&d.tw, g_na_tw)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&d.r2c, g_na_r2c)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&d.f, g_na_f)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&d.mat, g_na_mat)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&d.err, g_na_err)) != cudaSuccess)
      d.setup = e;
  });
  *out = &d;
  return d.setup;
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
  // square planes only (the three-pass kernels); the limit of the fixed scratch
  if (nx != ny || nx > kNaMax || nz > kNaMax) return RPM_ERR_UNSUPPORTED_GRID;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  // A call may copy host tables into the shared arrays; such copies cannot be
  // recorded into a graph (their source is this call's stack frame), so a
  // capturing stream is refused outright.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return RPM_ERR_INVALID_ARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return RPM_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaDevices) return RPM_ERR_CUDA;
  NaDevice* a = nullptr;
  if (na_setup(dev, &a) != cudaSuccess) return RPM_ERR_CUDA;

  const int nxh = nx / 2;
  float2 mat[2 * 256];
  std::memset(mat, 0, sizeof(mat));
  for (int i = 0; i < n_phases; ++i) {
    mat[i] = make_float2((float)(phases[i].lambda - c0.lambda), (float)(phases[i].mu - c0.mu));
    mat[256 + i] = make_float2((float)phases[i].lambda, (float)phases[i].mu);
  }
  {
    std::lock_guard<std::mutex> lk(a->mu);
    const bool same = a->have_key && a->key_grid[0] == nx && a->key_grid[1] == ny &&
                      a->key_grid[2] == nz && std::memcmp(a->key_mat, mat, sizeof(mat)) == 0;
    if (!same) {
      // host tables (the same definitions as a context's), then stream-ordered
      // copies into the file-scope arrays.  From pageable host memory a copy
      // returns once its source has been staged, so the stack arrays may go.
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
        f[nxh + 1 + s] =
            make_int2((2 * k < ny) ? k : k - ny, (ny % 2 == 0 && 2 * k == ny) ? 1 : 0);
      }
      a->have_key = false;
      if (cudaMemcpyAsync(a->tw, tw, sizeof(tw), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(a->r2c, r2c, sizeof(r2c), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(a->f, f, sizeof(f), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(a->mat, mat, sizeof(mat), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return RPM_ERR_CUDA;
      a->key_grid[0] = nx;
      a->key_grid[1] = ny;
      a->key_grid[2] = nz;
      std::memcpy(a->key_mat, mat, sizeof(mat));
      a->have_key = true;
    }
  }

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
  g.err = a->err;
  // the spectrum is fully written by the first pass before it is read: no clearing
  if (launch_apply_gamma(g, in, out, a->spec, E, flags, st) != cudaSuccess) return RPM_ERR_CUDA;
  return RPM_OK;
}
