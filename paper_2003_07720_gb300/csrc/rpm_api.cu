// Host side of the C ABI declared in include/rpm.h: the context (device
// buffers, FFT tables, material tables) and the solver loops of
// Algorithm 1 (basic scheme) and Algorithm 2 (RPM-FFT).
//
// Every field-sized step runs in the CUDA kernels of gamma_kernels.cu and
// field_kernels.cu; the host only sequences launches, takes the small
// decisions of Algorithm 2 (convergence, the one-or-two-vector rule of
// Eq. 3.8) and inverts the p x p matrix I - H in float64.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "fft_smem.cuh"
#include "rpm.h"
#include "rpm_internal.h"

using namespace rpm;

namespace {

constexpr int kPCap = kMaxBasis;      // largest basis the kernels accept
// layout of the small float64 device array
constexpr int kSums = 0;              // 1 + kPCap reduced sums
constexpr int kC = kSums + kPCap + 8;   // Newton correction c
constexpr int kRes = kC + kPCap;      // residual
constexpr int kBatch = 4;             // steps between host reads while the basis is empty
constexpr int kBatchMax = 16;         // longest batch when the decay rate predicts it
constexpr int kFields = 10;           // field buffers of a context (see rpm_ctx::fields)
constexpr int kMaxRebase = 16;        // re-centrings of one solve (see solve_impl)
// Basis growth is skipped while |xi^nu - xi^(nu-1)| < kGrowNoise |xi|: such a
// difference is dominated by the float32 rounding of F (about 2e-7 |xi|).
constexpr double kGrowNoise = 1e-5;
constexpr int kM = kRes + 8;          // (I - H)^-1, kPCap x kPCap
constexpr int kSmall = kM + kPCap * kPCap;
constexpr int kTicket = kSmall;       // one more slot: the fused reduction's counter
constexpr int kFusedMaxBlocks = 1024; // dots blocks up to which the fused reduction pays

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct rpm_ctx {
  rpm_grid grid{};
  rpm_options opt{};
  int p_cap = 0;
  cudaStream_t st = nullptr;
  std::vector<rpm_iso> phases;
  rpm_iso c0{};
  GridDev g{};
  GridDev gb{};                      // g with the Algorithm 3 pre-step table (s_b)
  float2* dmat_b = nullptr;          // per phase (alpha lam - beta lam0, alpha mu - beta mu0)
  float4* post = nullptr;            // per phase (lam_a, mu_a, k_s, h_s) of Algorithm 3
  GridDev gp{};                      // g with the table (-lam0, -mu0): compatible projection
  float2* dmat_p = nullptr;
  long long n = 0;
  size_t fsz = 0;                    // floats per field (6 n)
  size_t fst = 0;                    // stride between internal fields (6 n + pad)
  char* tables = nullptr;
  uint8_t* phase = nullptr;
  float2* spec = nullptr;
  float* fields = nullptr;           // eps[2], xi[3], D[2], eps_b, base, defect
  float* Z = nullptr;
  float* W = nullptr;
  double* partials = nullptr;
  int nblk = 0;
  double* dsmall = nullptr;
  double* hsmall = nullptr;          // pinned host mirror
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  size_t bytes = 0;
  std::string err;
  std::vector<double> H;             // host copy of H = Z^T F_u Z (row-major, p x p)
  int p = 0;
  // The basis held in Z and W after the last solve that had one: its size,
  // H, and the map it belongs to (F_u depends on the phases, the materials,
  // C0 and the scheme, not on the load E); options.share_basis starts the
  // next solve of the same map from it.
  int sb_p = 0;
  std::vector<double> sb_H;
  std::vector<double> sb_key;
  long long mat_version = 0;         // bumped by every phase or material change
  long long launches = 0;            // kernels launched by the current solve
  double proj_bytes = 0;             // algorithmic bytes of the projection kernels
  // event pairs for opt.profile: (start, stop, category 0 = Gamma0, 1 = projections);
  // groups seen and bracketed per category in the current solve
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_cat;
  size_t prof_used = 0;
  long long prof_seen[2] = {0, 0}, prof_rec[2] = {0, 0};
  // optional residual history (host arrays owned by the caller)
  double* trace_res = nullptr;
  int* trace_p = nullptr;
  int trace_cap = 0;
};

namespace {

bool ck(rpm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

rpm_status fail(rpm_ctx* c, rpm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

void build_twiddles(int L, std::vector<float2>& out) {
  const int N1 = split_n1(L), N2 = split_n2(L);
  for (int n2 = 0; n2 < N2; ++n2)
    for (int k1 = 0; k1 < N1; ++k1) {
      const double a = -2.0 * M_PI * (double)n2 * (double)k1 / (double)L;
      out.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
    }
}

bool valid_options(const rpm_options& o) {
  return o.n_max >= 1 && o.p_max >= 0 && o.p_max <= kPCap && o.max_iters >= 0 && o.tol >= 0 &&
         o.profile >= 0 &&
         o.t_ratio >= 0 && o.nyquist == RPM_NYQ_ZERO_MIXED && o.diverge_factor > 0 &&
         (o.scheme == RPM_SCHEME_BASIC || o.scheme == RPM_SCHEME_POLARIZATION) &&
         std::isfinite(o.alpha) && std::isfinite(o.beta) && std::isfinite(o.warm_tol) &&
         o.warm_c0_scale > 0 && o.warm_max_iters >= 0 && o.warm_p_max >= 0 &&
         o.warm_p_max <= kPCap && (o.warm_from_eps0 == 0 || o.warm_from_eps0 == 1) &&
         (o.autotune == 0 || o.autotune == 1) && o.plane_variant >= 0 &&
         o.plane_variant <= 2 && o.pencil_variant >= 0 && o.pencil_variant <= 3 &&
         (o.share_basis == 0 || o.share_basis == 1);
}

// Per-phase (lam - lam0, mu - mu0) for the polarization of pass A.
cudaError_t upload_dmat(rpm_ctx* c) {
  std::vector<float2> dm(256, make_float2(0.f, 0.f));
  for (size_t i = 0; i < c->phases.size(); ++i)
    dm[i] = make_float2((float)(c->phases[i].lambda - c->c0.lambda),
                        (float)(c->phases[i].mu - c->c0.mu));
  return cudaMemcpyAsync((void*)c->g.dmat, dm.data(), 256 * sizeof(float2),
                         cudaMemcpyHostToDevice, c->st);
}

cudaError_t upload_scheme_tables(rpm_ctx* c);

void set_variants(rpm_ctx* c, int plane_v, int pencil_t) {
  c->g.plane_v = c->gb.plane_v = c->gp.plane_v = plane_v;
  c->g.pencil_t = c->gb.pencil_t = c->gp.pencil_t = pencil_t;
}

// Tile autotuner: time one Gamma0 application (linear part, zeroed fields)
// with every distinct pair of plane-pass and z-pass variants on this
// context's grid, keep the fastest.
bool autotune_tiles(rpm_ctx* c) {
  float* in = c->fields;
  float* out = c->fields + c->fst;
  if (!ck(c, cudaMemsetAsync(in, 0, c->fsz * 4, c->st), "autotune") ||
      !ck(c, cudaMemsetAsync(c->spec, 0, (size_t)6 * c->g.nz * c->g.plane * sizeof(float2), c->st),
          "autotune"))
    return false;
  float best = 1e30f;
  int best_pl = 0, best_v = 0;
  std::vector<std::pair<int, int>> seen;   // (plane kernels, pencils per block; -1: fused z)
  for (int k = 0; k < 12; ++k) {
    GridDev g = c->g;
    g.plane_v = k / 4;
    g.pencil_t = k % 4;
    const std::pair<int, int> key(plane_variant(g), fused_z_pass(g) ? -1 : pencil_tile(g));
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
    seen.push_back(key);
    if (launch_apply_gamma(g, in, out, c->spec, nullptr, GM_LINEAR, c->st) != cudaSuccess) {
      cudaGetLastError();   // variant not available on this grid (shared memory)
      continue;
    }
    constexpr int kReps = 5;
    if (!ck(c, cudaEventRecord(c->ev0, c->st), "autotune")) return false;
    for (int r = 0; r < kReps; ++r)
      if (!ck(c, launch_apply_gamma(g, in, out, c->spec, nullptr, GM_LINEAR, c->st), "autotune"))
        return false;
    float ms = 0.f;
    if (!ck(c, cudaEventRecord(c->ev1, c->st), "autotune") ||
        !ck(c, cudaEventSynchronize(c->ev1), "autotune") ||
        !ck(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1), "autotune"))
      return false;
    if (ms < best) {
      best = ms;
      best_pl = g.plane_v;
      best_v = g.pencil_t;
    }
  }
  set_variants(c, best_pl, best_v);
  return true;
}

// Switch the reference medium C0 of the context (tables and Green operator).
cudaError_t set_reference_medium(rpm_ctx* c, rpm_iso c0) {
  c->c0 = c0;
  c->g.lam0 = c->gb.lam0 = c->gp.lam0 = (float)c0.lambda;
  c->g.mu0 = c->gb.mu0 = c->gp.mu0 = (float)c0.mu;
  cudaError_t e = upload_dmat(c);
  if (e != cudaSuccess) return e;
  return upload_scheme_tables(c);
}

// Algorithm 3 tables for the current options: s_b = alpha C:eps - beta C0:eps
// (isotropic per phase) and the post-step moduli.
cudaError_t upload_scheme_tables(rpm_ctx* c) {
  std::vector<float2> db(256, make_float2(0.f, 0.f));
  std::vector<float4> pt(256, make_float4(0.f, 0.f, 1.f, 1.f));
  const double a = c->opt.alpha, b = c->opt.beta, l0 = c->c0.lambda, m0 = c->c0.mu;
  // projection table: (C - C0) replaced by -C0 for every phase id
  std::vector<float2> dp(256, make_float2((float)-l0, (float)-m0));
  for (size_t i = 0; i < c->phases.size(); ++i) {
    const double l = c->phases[i].lambda, m = c->phases[i].mu;
    db[i] = make_float2((float)(a * l - b * l0), (float)(a * m - b * m0));
    const double ls = l + l0, ms = m + m0;   // C + C0
    pt[i] = make_float4((float)(l + (1.0 - b) * l0), (float)(m + (1.0 - b) * m0),
                        (float)(ls / (3.0 * ls + 2.0 * ms)), (float)(0.5 / ms));
  }
  cudaError_t e = cudaMemcpyAsync(c->dmat_b, db.data(), 256 * sizeof(float2),
                                  cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(c->post, pt.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(c->dmat_p, dp.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice, c->st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->st);
}

// Gauss-Jordan inverse with partial pivoting (p <= 32), float64.
bool invert(int p, const std::vector<double>& A, std::vector<double>& inv) {
  std::vector<double> a(A);
  inv.assign((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i) inv[(size_t)i * p + i] = 1.0;
  for (int col = 0; col < p; ++col) {
    int piv = col;
    for (int r = col + 1; r < p; ++r)
      if (std::fabs(a[(size_t)r * p + col]) > std::fabs(a[(size_t)piv * p + col])) piv = r;
    const double pv = a[(size_t)piv * p + col];
    if (!(std::fabs(pv) > 1e-300)) return false;
    if (piv != col)
      for (int k = 0; k < p; ++k) {
        std::swap(a[(size_t)piv * p + k], a[(size_t)col * p + k]);
        std::swap(inv[(size_t)piv * p + k], inv[(size_t)col * p + k]);
      }
    const double ip = 1.0 / pv;
    for (int k = 0; k < p; ++k) {
      a[(size_t)col * p + k] *= ip;
      inv[(size_t)col * p + k] *= ip;
    }
    for (int r = 0; r < p; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * p + col];
      if (f == 0.0) continue;
      for (int k = 0; k < p; ++k) {
        a[(size_t)r * p + k] -= f * a[(size_t)col * p + k];
        inv[(size_t)r * p + k] -= f * inv[(size_t)col * p + k];
      }
    }
  }
  return true;
}

void upload_materials(rpm_ctx* c, std::vector<float2>& dm, std::vector<float2>& cm) {
  dm.clear();
  cm.clear();
  for (const auto& ph : c->phases) {
    dm.push_back(make_float2((float)(ph.lambda - c->c0.lambda), (float)(ph.mu - c->c0.mu)));
    cm.push_back(make_float2((float)ph.lambda, (float)ph.mu));
  }
}

// --- thin wrappers that record the failing step ---------------------------
struct Ops {
  rpm_ctx* c;
  // optional event bracket around a group of launches (opt.profile)
  size_t mark(int cat) {
    if (!c->opt.profile) return (size_t)-1;
    if (c->prof_seen[cat]++ % c->opt.profile != 0) return (size_t)-1;   // every k-th group
    if (c->prof_used * 2 + 2 > c->prof_ev.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return (size_t)-1;
      c->prof_ev.push_back(a);
      c->prof_ev.push_back(b);
      c->prof_cat.push_back(cat);
    }
    const size_t i = c->prof_used++;
    c->prof_cat[i] = cat;
    ++c->prof_rec[cat];
    cudaEventRecord(c->prof_ev[2 * i], c->st);
    return i;
  }
  void done(size_t i) {
    if (i != (size_t)-1) cudaEventRecord(c->prof_ev[2 * i + 1], c->st);
  }
  bool gamma(const float* in, float* out, const double* E, int mode, const float* add = nullptr) {
    const size_t m = mark(0);
    c->launches += gamma_add_launches(c->g, out, add, c->spec);
    const bool ok =
        ck(c, launch_apply_gamma(c->g, in, out, c->spec, E, mode, c->st, add), "apply_gamma");
    done(m);
    return ok;
  }
  // the solver's fixed-point map F (linear: F_u, i.e. E = 0)
  bool fmap(const float* in, float* out, const double* E, bool linear) {
    if (c->opt.scheme == RPM_SCHEME_BASIC) return gamma(in, out, E, linear ? GM_LINEAR : GM_FULL_MAP);
    const size_t m = mark(0);
    c->launches += polarization_launches(c->gb, in, out, c->spec);
    float* eb = c->fields + 7 * c->fst;
    double Eb[6] = {0, 0, 0, 0, 0, 0};
    if (!linear)
      for (int k = 0; k < 6; ++k) Eb[k] = c->opt.beta * E[k];
    const bool ok = ck(c, launch_polarization_map(c->gb, c->post, in, eb, out, c->spec, Eb,
                                                  linear ? GM_LINEAR : GM_FULL_MAP, c->st),
                       "polarization map");
    done(m);
    return ok;
  }
  // sums[0..K] <- dots of x against Y (see launch_dots)
  // sums[0..K] <- dots (see launch_dots); with M, also the Newton step into c
  // and the residual.  K <= 32 on grids up to ~100^3: one fused launch (the
  // last block's serial tail costs more than two launches beyond that)
  bool dots(const float* x, const float* xm, const float* Y, int K, double* sums,
            const double* M = nullptr, double* cN = nullptr, double* res = nullptr,
            double inv_norm = 0.0) {
    const size_t m = mark(1);
    c->proj_bytes += (double)(K + 1 + (xm ? 1 : 0)) * (double)c->fsz * 4.0;
    bool ok;
    if (K <= 32 && c->nblk <= kFusedMaxBlocks) {
      c->launches += 1;
      ok = ck(c, launch_dots_fused(x, xm, Y, (long long)c->fst, K, c->n, c->partials, c->nblk,
                                   sums, reinterpret_cast<unsigned int*>(c->dsmall + kTicket), M,
                                   cN, res, inv_norm, c->st),
              "dots");
    } else {
      c->launches += 1 + dots_launches(K) + (M ? 1 : 0);
      ok = ck(c, launch_dots(x, xm, Y, (long long)c->fst, K, c->n, c->partials, c->nblk, c->st),
              "dots") &&
           ck(c, launch_reduce_partials(c->partials, c->nblk, K + 1, sums, c->st), "reduce") &&
           (!M || ck(c, launch_newton(sums, K, M, cN, res, inv_norm, c->st), "newton"));
    }
    done(m);
    return ok;
  }
  bool combine(float* out, const float* x, float xs, const float* Y, int K, const double* coef,
               float cscale) {
    const size_t m = mark(1);
    c->launches += combine_launches(K);
    c->proj_bytes += (double)(K + (x ? 1 : 0) + 1) * (double)c->fsz * 4.0;
    const bool ok =
        ck(c, launch_combine(out, x, xs, Y, (long long)c->fst, K, coef, cscale, c->n, c->st),
           "combine");
    done(m);
    return ok;
  }
  bool read_small(int off, int count) {
    if (!ck(c, cudaMemcpyAsync(c->hsmall + off, c->dsmall + off, sizeof(double) * count,
                               cudaMemcpyDeviceToHost, c->st),
            "read"))
      return false;
    return ck(c, cudaStreamSynchronize(c->st), "sync");
  }
};

}  // namespace

extern "C" {

void rpm_default_options(rpm_options* o) {
  if (!o) return;
  o->n_max = 10;
  o->p_max = 20;
  o->max_iters = 5000;
  o->tol = 1e-6;
  o->t_ratio = 0.1;
  o->nyquist = RPM_NYQ_ZERO_MIXED;
  o->diverge_factor = 1e10;
  o->max_device_gb = 0.0;
  o->profile = 0;
  o->scheme = RPM_SCHEME_BASIC;
  o->alpha = 2.0;
  o->beta = 2.0;
  o->warm_tol = 0.0;
  o->warm_c0_scale = 1.0;
  o->warm_max_iters = 2000;
  o->warm_p_max = 0;
  o->warm_from_eps0 = 0;
  o->autotune = 0;
  o->plane_variant = 0;
  o->pencil_variant = 0;
  o->share_basis = 0;
}

int rpm_grid_supported(int nx, int ny, int nz) { return grid_supported(nx, ny, nz) ? 1 : 0; }

const char* rpm_status_string(rpm_status s) {
  switch (s) {
    case RPM_OK: return "RPM_OK";
    case RPM_ERR_INVALID_ARG: return "RPM_ERR_INVALID_ARG";
    case RPM_ERR_UNSUPPORTED_GRID: return "RPM_ERR_UNSUPPORTED_GRID";
    case RPM_ERR_OOM: return "RPM_ERR_OOM";
    case RPM_ERR_CUDA: return "RPM_ERR_CUDA";
    case RPM_ERR_NOT_CONVERGED: return "RPM_ERR_NOT_CONVERGED";
    case RPM_ERR_DIVERGED: return "RPM_ERR_DIVERGED";
    case RPM_ERR_TIMEOUT: return "RPM_ERR_TIMEOUT";
  }
  return "RPM_ERR_UNKNOWN";
}

const char* rpm_last_error(const rpm_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t rpm_device_bytes(const rpm_ctx* c) { return c ? c->bytes : 0; }

}  // extern "C"

bool rpm::ctx_cell_view(const rpm_ctx* c, CellView* v) {
  if (!c || !v || c->phases.empty()) return false;
  v->nx = c->grid.nx;
  v->ny = c->grid.ny;
  v->nz = c->grid.nz;
  v->phase = c->phase;
  v->phases = c->phases.data();
  v->n_phases = (int)c->phases.size();
  v->st = c->st;
  return true;
}

extern "C" {

void rpm_destroy(rpm_ctx* c) {
  if (!c) return;
  cudaFree(c->tables);
  cudaFree(c->phase);
  cudaFree(c->spec);
  cudaFree(c->fields);
  cudaFree(c->Z);
  cudaFree(c->W);
  cudaFree(c->partials);
  cudaFree(c->dsmall);
  if (c->hsmall) cudaFreeHost(c->hsmall);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  delete c;
}

rpm_status rpm_set_phase(rpm_ctx* c, const uint8_t* phase, int on_device) {
  if (!c || !phase) return fail(c, RPM_ERR_INVALID_ARG, "null argument");
  if (!on_device) {   // largest id by a branch-free (vectorisable) reduction
    uint8_t mx = 0;
    for (long long i = 0; i < c->n; ++i) mx = phase[i] > mx ? phase[i] : mx;
    if (c->n > 0 && mx >= c->phases.size())
      return fail(c, RPM_ERR_INVALID_ARG, "phase id out of range");
  }
  if (!ck(c, cudaMemcpyAsync(c->phase, phase, (size_t)c->n,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st),
          "phase upload"))
    return RPM_ERR_CUDA;
  ++c->mat_version;   // a stored basis belongs to the previous cell
  return RPM_OK;
}

rpm_status rpm_set_options(rpm_ctx* c, const rpm_options* o) {
  if (!c || !o) return fail(c, RPM_ERR_INVALID_ARG, "null argument");
  if (!valid_options(*o) || o->p_max > c->p_cap)
    return fail(c, RPM_ERR_INVALID_ARG, "invalid options (p_max above the creation value?)");
  const bool keep_tuned = c->opt.autotune && o->autotune;
  c->opt = *o;
  c->g.nyquist = o->nyquist;
  c->gb.nyquist = c->gp.nyquist = o->nyquist;
  if (!keep_tuned) set_variants(c, o->plane_variant, o->pencil_variant);
  if (!ck(c, upload_scheme_tables(c), "scheme tables")) return RPM_ERR_CUDA;
  return RPM_OK;
}

rpm_status rpm_create(const rpm_grid* grid, const uint8_t* phase, int phase_on_device, int n_phases,
                      const rpm_iso* phases, rpm_iso c0, const rpm_options* opt, void* stream,
                      rpm_ctx** out) {
  if (!out) return RPM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid || !phase || !phases || n_phases < 1 || n_phases > 256) return RPM_ERR_INVALID_ARG;
  rpm_options o;
  rpm_default_options(&o);
  if (opt) o = *opt;
  if (!valid_options(o)) return RPM_ERR_INVALID_ARG;
  if (!(c0.mu > 0) || !(c0.lambda + 2 * c0.mu > 0)) return RPM_ERR_INVALID_ARG;
  if (!grid_supported(grid->nx, grid->ny, grid->nz)) return RPM_ERR_UNSUPPORTED_GRID;

  rpm_ctx* c = new rpm_ctx();
  c->grid = *grid;
  c->opt = o;
  c->p_cap = o.p_max;
  c->st = (cudaStream_t)stream;
  c->phases.assign(phases, phases + n_phases);
  c->c0 = c0;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz, nxh = nx / 2;
  c->n = (long long)nx * ny * nz;
  c->fsz = (size_t)6 * c->n;
  // Internal fields sit 6 n floats + 4352 bytes apart: equal power-of-two-like
  // strides put the 2p concurrent basis streams of the projections on the same
  // DRAM channels.
  c->fst = c->fsz + 1088;
  GridDev& g = c->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxh = nxh;
  g.n = c->n;
  g.plane = ny * (nxh + 1);
  g.n_phases = n_phases;
  g.lam0 = (float)c0.lambda;
  g.mu0 = (float)c0.mu;
  g.inv_lx = (float)(1.0 / (grid->lx > 0 ? grid->lx : 1.0));
  g.inv_ly = (float)(1.0 / (grid->ly > 0 ? grid->ly : 1.0));
  g.inv_lz = (float)(1.0 / (grid->lz > 0 ? grid->lz : 1.0));
  g.nyquist = o.nyquist;

  // host tables
  std::vector<float2> twx, twy, twz, r2c, dm, cm;
  build_twiddles(nxh, twx);
  build_twiddles(ny, twy);
  build_twiddles(nz, twz);
  for (int k = 0; k <= nxh; ++k) {
    const double a = -2.0 * M_PI * (double)k / (double)nx;
    r2c.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
  }
  std::vector<int2> fx, fy;
  for (int s = 0; s <= nxh; ++s) {
    const int k = s < nxh ? freq_of_rt(nxh, s) : nxh;
    const bool nyq = (k == nxh);
    fx.push_back(make_int2(nyq ? -k : k, nyq ? 1 : 0));
  }
  for (int s = 0; s < ny; ++s) {
    const int k = freq_of_rt(ny, s);
    const int m = (2 * k < ny) ? k : k - ny;
    fy.push_back(make_int2(m, (ny % 2 == 0 && ny > 1 && 2 * k == ny) ? 1 : 0));
  }
  upload_materials(c, dm, cm);

  // sizes
  size_t off = 0;
  const size_t o_twx = off; off = align_up(off + twx.size() * 8, 256);
  const size_t o_twy = off; off = align_up(off + twy.size() * 8, 256);
  const size_t o_twz = off; off = align_up(off + twz.size() * 8, 256);
  const size_t o_r2c = off; off = align_up(off + r2c.size() * 8, 256);
  const size_t o_fx = off; off = align_up(off + fx.size() * 8, 256);
  const size_t o_fy = off; off = align_up(off + fy.size() * 8, 256);
  const size_t o_dm = off; off = align_up(off + 256 * 8, 256);
  const size_t o_cm = off; off = align_up(off + 256 * 8, 256);
  const size_t o_db = off; off = align_up(off + 256 * 8, 256);
  const size_t o_pt = off; off = align_up(off + 256 * 16, 256);
  const size_t o_dp = off; off = align_up(off + 256 * 8, 256);
  const size_t o_err = off; off = align_up(off + 16, 256);
  const size_t tab_bytes = off;
  c->nblk = std::max(dots_blocks_for(c->n), stress_blocks_for(c->n));
  const size_t fbytes = c->fst * sizeof(float);
  const size_t spec_bytes = (size_t)6 * nz * g.plane * sizeof(float2);
  const size_t need = tab_bytes + align_up((size_t)c->n, 256) + spec_bytes + kFields * fbytes +
                      2 * (size_t)c->p_cap * fbytes + (size_t)(kPCap + 1) * c->nblk * 8 +
                      (kSmall + 1) * 8;
  if (o.max_device_gb > 0 && (double)need > o.max_device_gb * 1e9) {
    rpm_destroy(c);
    return RPM_ERR_OOM;
  }
  auto alloc = [&](void** p, size_t b) {
    if (b == 0) b = 256;
    cudaError_t e = cudaMalloc(p, b);
    if (e == cudaSuccess) c->bytes += b;
    return e;
  };
  cudaError_t e = cudaSuccess;
  if ((e = alloc((void**)&c->tables, tab_bytes)) != cudaSuccess ||
      (e = alloc((void**)&c->phase, align_up((size_t)c->n, 256))) != cudaSuccess ||
      (e = alloc((void**)&c->spec, spec_bytes)) != cudaSuccess ||
      (e = alloc((void**)&c->fields, kFields * fbytes)) != cudaSuccess ||
      (e = alloc((void**)&c->Z, (size_t)c->p_cap * fbytes)) != cudaSuccess ||
      (e = alloc((void**)&c->W, (size_t)c->p_cap * fbytes)) != cudaSuccess ||
      (e = alloc((void**)&c->partials, (size_t)(kPCap + 1) * c->nblk * 8)) != cudaSuccess ||
      (e = alloc((void**)&c->dsmall, (kSmall + 1) * 8)) != cudaSuccess) {
    cudaGetLastError();
    rpm_destroy(c);
    return e == cudaErrorMemoryAllocation ? RPM_ERR_OOM : RPM_ERR_CUDA;
  }
  if (cudaMallocHost((void**)&c->hsmall, kSmall * 8) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    rpm_destroy(c);
    return RPM_ERR_CUDA;
  }
  char* t = c->tables;
  auto put = [&](size_t o2, const void* src, size_t b) {
    return cudaMemcpyAsync(t + o2, src, b, cudaMemcpyHostToDevice, c->st);
  };
  std::vector<float2> dm256(256, make_float2(0.f, 0.f)), cm256(256, make_float2(0.f, 0.f));
  for (int i = 0; i < n_phases; ++i) {
    dm256[i] = dm[i];
    cm256[i] = cm[i];
  }
  if (put(o_twx, twx.data(), twx.size() * 8) != cudaSuccess ||
      put(o_twy, twy.data(), twy.size() * 8) != cudaSuccess ||
      put(o_twz, twz.data(), twz.size() * 8) != cudaSuccess ||
      put(o_r2c, r2c.data(), r2c.size() * 8) != cudaSuccess ||
      put(o_fx, fx.data(), fx.size() * 8) != cudaSuccess ||
      put(o_fy, fy.data(), fy.size() * 8) != cudaSuccess ||
      put(o_dm, dm256.data(), 256 * 8) != cudaSuccess ||
      put(o_cm, cm256.data(), 256 * 8) != cudaSuccess ||
      cudaMemsetAsync(c->dsmall, 0, (kSmall + 1) * 8, c->st) != cudaSuccess ||
      cudaMemsetAsync(t + o_err, 0, 16, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    rpm_destroy(c);
    return RPM_ERR_CUDA;
  }
  g.tw_x = (const float2*)(t + o_twx);
  g.tw_y = (const float2*)(t + o_twy);
  g.tw_z = (const float2*)(t + o_twz);
  g.r2c_w = (const float2*)(t + o_r2c);
  g.fx = (const int2*)(t + o_fx);
  g.fy = (const int2*)(t + o_fy);
  g.dmat = (const float2*)(t + o_dm);
  g.cmat = (const float2*)(t + o_cm);
  g.phase = c->phase;
  g.err = (int*)(t + o_err);
  c->dmat_b = (float2*)(t + o_db);
  c->post = (float4*)(t + o_pt);
  c->dmat_p = (float2*)(t + o_dp);
  c->gb = g;
  c->gb.dmat = c->dmat_b;
  c->gp = g;
  c->gp.dmat = c->dmat_p;
  set_variants(c, o.plane_variant, o.pencil_variant);
  if (!ck(c, upload_scheme_tables(c), "scheme tables")) {
    rpm_destroy(c);
    return RPM_ERR_CUDA;
  }
  rpm_status s = rpm_set_phase(c, phase, phase_on_device);
  if (s == RPM_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = RPM_ERR_CUDA;
  if (s == RPM_OK && o.autotune && !autotune_tiles(c)) s = RPM_ERR_CUDA;
  if (s != RPM_OK) {
    rpm_destroy(c);
    return s;
  }
  *out = c;
  return RPM_OK;
}

int rpm_pencil_tile(const rpm_ctx* c) { return c ? pencil_tile(c->g) : 0; }

int rpm_plane_variant(const rpm_ctx* c) { return c ? plane_variant(c->g) : -1; }

rpm_status rpm_bounded_wait_check(void* cuda_stream, int* gave_up, float* waited_ms) {
  if (!gave_up || !waited_ms) return RPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int h = 0;
  float ms = 0.f;
  bool ok = cudaMalloc(&d, sizeof(int)) == cudaSuccess &&
            cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess &&
            cudaMemsetAsync(d, 0, sizeof(int), st) == cudaSuccess &&
            cudaEventRecord(a, st) == cudaSuccess && launch_wait_selfcheck(d, st) == cudaSuccess &&
            cudaEventRecord(b, st) == cudaSuccess &&
            cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (d) cudaFree(d);
  if (!ok) return RPM_ERR_CUDA;
  *gave_up = h;
  *waited_ms = ms;
  return RPM_OK;
}

rpm_status rpm_set_trace(rpm_ctx* c, double* residuals, int* basis_sizes, int capacity) {
  if (!c || capacity < 0) return fail(c, RPM_ERR_INVALID_ARG, "bad trace arguments");
  c->trace_res = residuals;
  c->trace_p = basis_sizes;
  c->trace_cap = capacity;
  return RPM_OK;
}

rpm_status rpm_apply_gamma(rpm_ctx* c, const float* in, const double E[6], float* out, int flags) {
  if (!c || !in || !out) return fail(c, RPM_ERR_INVALID_ARG, "null argument");
  if (flags < RPM_GAMMA_FULL_MAP || flags > RPM_GAMMA_PROJECT)
    return fail(c, RPM_ERR_INVALID_ARG, "bad flags");
  if ((flags == RPM_GAMMA_FULL_MAP || flags == RPM_GAMMA_PROJECT) && !E)
    return fail(c, RPM_ERR_INVALID_ARG, "E required");
  if (in == out) return fail(c, RPM_ERR_INVALID_ARG, "in and out alias");
  if (flags == RPM_GAMMA_PROJECT) {
    // E - Gamma0 * ((-C0) : in) = E + Gamma0 * (C0 : in): the pass-A table of gp
    c->launches += gamma_launches(c->g);
    if (!ck(c, launch_apply_gamma(c->gp, in, out, c->spec, E, GM_FULL_MAP, c->st), "project"))
      return RPM_ERR_CUDA;
    return RPM_OK;
  }
  Ops ops{c};
  if (!ops.gamma(in, out, E, flags)) return RPM_ERR_CUDA;
  return RPM_OK;
}

}  // extern "C"

namespace {

// Everything F_u depends on besides the grid: phases and materials (by
// version), C0, the scheme and its parameters, the Nyquist rule.
std::vector<double> basis_key(const rpm_ctx* c) {
  return {(double)c->mat_version, c->c0.lambda, c->c0.mu, (double)c->opt.scheme, c->opt.alpha,
          c->opt.beta, (double)c->opt.nyquist};
}

// One solve of Algorithm 2 (Algorithm 1 when p_max = 0).
rpm_status solve_impl(rpm_ctx* c, const double E[6], const float* eps0, float* eps_out,
                      float* sig_out, int out_on_host, rpm_solve_info* info) {
  Ops ops{c};
  const rpm_options& o = c->opt;
  const size_t F = c->fst;
  float* epsb[2] = {c->fields, c->fields + F};
  float* xi[3] = {c->fields + 2 * F, c->fields + 3 * F, c->fields + 4 * F};
  float* D[2] = {c->fields + 5 * F, c->fields + 6 * F};
  double* ds = c->dsmall;
  double* hs = c->hsmall;
  double En2 = 0;
  for (int k = 0; k < 6; ++k) En2 += (k < 3 ? 1.0 : 2.0) * E[k] * E[k];
  const double inv_norm = 1.0 / ((En2 > 0 ? std::sqrt(En2) : 1.0) * std::sqrt((double)c->n));

  rpm_solve_info inf{};
  inf.status = RPM_OK;
  c->p = 0;
  c->launches = 0;
  c->proj_bytes = 0;
  c->prof_used = 0;
  c->prof_seen[0] = c->prof_seen[1] = c->prof_rec[0] = c->prof_rec[1] = 0;
  c->H.clear();
  std::vector<double> M;

  if (!ck(c, cudaEventRecord(c->ev0, c->st), "event")) return RPM_ERR_CUDA;
  if (!ck(c, cudaMemsetAsync(ds, 0, (kSmall + 1) * 8, c->st), "memset")) return RPM_ERR_CUDA;
  // A basis of the same map left in Z and W by an earlier solve (another load
  // E, or the same one): with share_basis the solve starts from its leading
  // min(size, p_max) vectors, H's leading block and M = (I - H)^-1.
  const std::vector<double> key = basis_key(c);
  if (o.share_basis && c->sb_p > 0 && c->sb_key == key) {
    const int p = std::min(c->sb_p, std::min(o.p_max, c->p_cap));
    c->H.assign((size_t)p * p, 0.0);
    std::vector<double> A((size_t)p * p);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        c->H[(size_t)i * p + j] = c->sb_H[(size_t)i * c->sb_p + j];
        A[(size_t)i * p + j] = (i == j ? 1.0 : 0.0) - c->H[(size_t)i * p + j];
      }
    if (p > 0 && invert(p, A, M)) {
      if (!ck(c, cudaMemcpyAsync(ds + kM, M.data(), sizeof(double) * p * p,
                                 cudaMemcpyHostToDevice, c->st),
              "upload M"))
        return RPM_ERR_CUDA;
      c->p = p;
      inf.basis_reused = p;
    } else {
      c->H.clear();
    }
  }
  float* eps_cur = epsb[0];
  if (eps0) {
    if (!ck(c, cudaMemcpyAsync(eps_cur, eps0, c->fsz * 4, cudaMemcpyDeviceToDevice, c->st), "eps0"))
      return RPM_ERR_CUDA;
  } else if (++c->launches, !ck(c, launch_fill(eps_cur, E, c->n, c->st), "fill")) {
    return RPM_ERR_CUDA;
  }
  int cur = 0, hist = 1, it = 0, nu = 0, nF = 0;
  if (!ops.fmap(eps_cur, xi[0], E, false)) return RPM_ERR_CUDA;
  nF = 1;

  // Re-centring (defect correction).  After a stall the iterate is split as
  // eps = base + y, base frozen; the map is then y -> r + F_u y with the
  // defect r = F(base) - base, the same linear part (basis, H and M stay
  // valid) and a fixed point at the same eps.  Float32 rounding then scales
  // with |y| instead of |eps|, which removes the float32 floor the plain
  // iteration meets on high-contrast cells.
  float* base = c->fields + 8 * F;
  float* defect = c->fields + 9 * F;
  bool based = false;
  int rebases = 0;
  auto step_map = [&](const float* in, float* out) -> bool {
    if (!based) return ops.fmap(in, out, E, false);
    // Eq. 3.9: the defect is added in the map's last pass
    if (o.scheme == RPM_SCHEME_BASIC) return ops.gamma(in, out, nullptr, GM_LINEAR, defect);
    if (!ops.fmap(in, out, nullptr, true)) return false;
    ++c->launches;
    return ck(c, launch_axpby(out, 1.f, out, 1.f, defect, c->n, c->st), "defect");
  };

  // residual, zeta - z = Z^T (xi - eps) and the Newton correction for the current pair (eps, xi)
  // (read = false: leave the residual on the device; the Newton correction is
  // all the next step needs)
  auto eval = [&](double& r, bool read = true) -> bool {
    if (!ops.dots(xi[cur], eps_cur, c->Z, c->p, ds + kSums, ds + kM, ds + kC, ds + kRes,
                  inv_norm))
      return false;
    if (!read) return true;
    if (!ops.read_small(kRes, 1)) return false;
    r = hs[kRes];
    return true;
  };

  // In(q, Z) of Algorithm 2 with the QR rule of Eq. 3.8.
  bool want_rebase = false;
  auto grow = [&]() -> bool {
    const int prev = (cur + 2) % 3, prev2 = (cur + 1) % 3;
    double* one = ds + kSums;   // scratch sums
    // D0 = xi^nu - xi^(nu-1), D1 = xi^(nu-1) - xi^(nu-2)
    if (!ck(c, (++c->launches, launch_axpby)(D[0], 1.f, xi[cur], -1.f, xi[prev], c->n, c->st), "axpby") ||
        !ck(c, (++c->launches, launch_axpby)(D[1], 1.f, xi[prev], -1.f, xi[prev2], c->n, c->st), "axpby"))
      return false;
    // Q-projection (classical Gram-Schmidt, twice)
    for (int pass = 0; pass < 2 && c->p > 0; ++pass)
      for (int k = 0; k < 2; ++k) {
        if (!ops.dots(D[k], nullptr, c->Z, c->p, one)) return false;
        if (!ops.combine(D[k], D[k], 1.f, c->Z, c->p, one + 1, -1.f)) return false;
      }
    // QR of [D0, D1]
    if (!ops.dots(D[1], nullptr, D[0], 1, ds + kSums)) return false;   // |D1|^2, <D1,D0>
    if (!ops.read_small(kSums, 2)) return false;
    const double n11 = hs[kSums], d10 = hs[kSums + 1];
    if (!ops.dots(D[0], nullptr, nullptr, 0, ds + kSums)) return false;
    if (!ops.read_small(kSums, 1)) return false;
    const double T11 = std::sqrt(std::max(hs[kSums], 0.0));
    if (!(T11 > 0) || !std::isfinite(T11)) return true;
    if (!ops.dots(xi[cur], nullptr, nullptr, 0, ds + kSums)) return false;
    if (!ops.read_small(kSums, 1)) return false;
    if (T11 < kGrowNoise * std::sqrt(std::max(hs[kSums], 0.0))) {   // rounding noise:
      want_rebase = true;   // re-centre, then grow from differences in the new coordinates
      return true;
    }
    const double T12 = d10 / T11;
    (void)n11;
    if (!ck(c, (++c->launches, launch_axpby)(D[1], 1.f, D[1], (float)(-T12 / T11), D[0], c->n, c->st), "axpby"))
      return false;
    if (!ops.dots(D[1], nullptr, nullptr, 0, ds + kSums)) return false;
    if (!ops.read_small(kSums, 1)) return false;
    const double T22 = std::sqrt(std::max(hs[kSums], 0.0));
    int ncand = 1;
    double Tn[2] = {T11, T22};
    if (std::fabs(T22) > o.t_ratio * std::fabs(T11)) ncand = 2;
    const int p_old = c->p;
    const int p_lim = std::min(o.p_max, c->p_cap);
    for (int k = 0; k < ncand && c->p < p_lim; ++k) {
      float* u = D[k];
      if (!(Tn[k] > 0)) continue;
      if (!ck(c, (++c->launches, launch_axpby)(u, (float)(1.0 / Tn[k]), u, 0.f, nullptr, c->n, c->st), "axpby"))
        return false;
      for (int pass = 0; pass < 2 && c->p > 0; ++pass) {
        if (!ops.dots(u, nullptr, c->Z, c->p, one)) return false;
        if (!ops.combine(u, u, 1.f, c->Z, c->p, one + 1, -1.f)) return false;
      }
      if (!ops.dots(u, nullptr, nullptr, 0, ds + kSums)) return false;
      if (!ops.read_small(kSums, 1)) return false;
      const double nu_ = std::sqrt(std::max(hs[kSums], 0.0));
      if (!(nu_ > 1e-10)) continue;
      float* zp = c->Z + (size_t)c->p * F;
      if (!ck(c, (++c->launches, launch_axpby)(zp, (float)(1.0 / nu_), u, 0.f, nullptr, c->n, c->st), "axpby"))
        return false;
      if (!ops.fmap(zp, c->W + (size_t)c->p * F, nullptr, true)) return false;
      ++nF;
      ++c->p;
    }
    const int p = c->p;
    if (p == p_old) return true;
    // extend H: H_ij = <Z_i, F_u Z_j>
    std::vector<double> Hn((size_t)p * p, 0.0);
    for (int i = 0; i < p_old; ++i)
      for (int j = 0; j < p_old; ++j) Hn[(size_t)i * p + j] = c->H[(size_t)i * p_old + j];
    for (int q = p_old; q < p; ++q) {
      if (!ops.dots(c->W + (size_t)q * F, nullptr, c->Z, p, ds + kSums)) return false;
      if (!ops.read_small(kSums, p + 1)) return false;
      for (int i = 0; i < p; ++i) Hn[(size_t)i * p + q] = hs[kSums + 1 + i];
      if (!ops.dots(c->Z + (size_t)q * F, nullptr, c->W, p, ds + kSums)) return false;
      if (!ops.read_small(kSums, p + 1)) return false;
      for (int j = 0; j < p; ++j) Hn[(size_t)q * p + j] = hs[kSums + 1 + j];
    }
    c->H = Hn;
    std::vector<double> A((size_t)p * p);
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) A[(size_t)i * p + j] = (i == j ? 1.0 : 0.0) - Hn[(size_t)i * p + j];
    if (!invert(p, A, M)) {
      c->err = "I - H is singular";
      return false;
    }
    if (!ck(c, cudaMemcpyAsync(ds + kM, M.data(), sizeof(double) * p * p, cudaMemcpyHostToDevice,
                               c->st),
            "upload M"))
      return false;
    return true;
  };

  auto trace = [&](int k, double rr) {
    if (c->trace_res && k < c->trace_cap) c->trace_res[k] = rr;
    if (c->trace_p && k < c->trace_cap) c->trace_p[k] = c->p;
  };
  // base += y; every stored xi -= y (coordinates of the new base); y = 0;
  // the defect is the current xi.  The residual is unchanged.
  auto rebase = [&]() -> bool {
    c->launches += 1;
    const bool ok_base = based ? ck(c, launch_axpby(base, 1.f, base, 1.f, eps_cur, c->n, c->st), "base")
                               : ck(c, cudaMemcpyAsync(base, eps_cur, c->fsz * 4,
                                                       cudaMemcpyDeviceToDevice, c->st), "base");
    if (!ok_base) return false;
    for (int k = 0; k < 3; ++k) {
      if (xi[k] == eps_cur) continue;
      ++c->launches;
      if (!ck(c, launch_axpby(xi[k], 1.f, xi[k], -1.f, eps_cur, c->n, c->st), "shift")) return false;
    }
    if (!ck(c, cudaMemsetAsync(eps_cur, 0, c->fsz * 4, c->st), "zero") ||
        !ck(c, cudaMemcpyAsync(defect, xi[cur], c->fsz * 4, cudaMemcpyDeviceToDevice, c->st),
            "defect"))
      return false;
    based = true;
    ++rebases;
    hist = 1;   // growth waits for differences of iterates in the new coordinates
    return true;
  };

  double r = 0;
  if (!eval(r)) return RPM_ERR_CUDA;
  trace(0, r);
  const double r0 = r;
  double r_best = r;
  int it_best = 0;
  double r_prev = r;   // residual and step of the previous host read
  int it_prev = 0;
  inf.residual0 = r0;
  rpm_status status = RPM_OK;
  for (;;) {
    if (!std::isfinite(r) || r > o.diverge_factor * r0) {
      status = RPM_ERR_DIVERGED;
      break;
    }
    if (r <= o.tol) break;
    if (it >= o.max_iters) {
      status = RPM_ERR_NOT_CONVERGED;
      break;
    }
    // Steps between host reads of the residual: up to kBatch while the basis
    // is empty, and with a basis while the residual is still far (> 100 tol)
    // from the test and no residual history is recorded, never past a
    // basis-growth point or max_iters.
    int batch = 1;
    if (c->p == 0 || (r > 1e2 * o.tol && !c->trace_res)) {
      batch = kBatch;
      // Predictive batching: with the residual falling geometrically at the
      // rate seen since the last read, a batch ends before the step that
      // would meet tol, so no step runs past it (one host read per batch).
      if (!c->trace_res && it > it_prev && r_prev > r && r > o.tol) {
        const double rate = std::pow(r / r_prev, 1.0 / (double)(it - it_prev));
        const double to_tol = std::log(o.tol / r) / std::log(rate);
        if (std::isfinite(to_tol) && to_tol > 1.0)
          batch = std::max(batch, std::min(kBatchMax, (int)(0.8 * to_tol)));
      }
      if (c->p < std::min(o.p_max, c->p_cap)) batch = std::min(batch, o.n_max + 1 - nu);
      batch = std::max(1, std::min(batch, o.max_iters - it));
    }
    r_prev = r;
    it_prev = it;
    for (int b = 0; b < batch; ++b) {
      float* eps_next;
      if (c->p == 0) {
        eps_next = xi[cur];
      } else {
        eps_next = (eps_cur == epsb[0]) ? epsb[1] : epsb[0];
        if (!ops.combine(eps_next, xi[cur], 1.f, c->Z, c->p, ds + kC, 1.f)) return RPM_ERR_CUDA;
      }
      const int nxt = (cur + 1) % 3;
      if (!step_map(eps_next, xi[nxt])) return RPM_ERR_CUDA;
      ++nF;
      ++it;
      ++nu;
      cur = nxt;
      hist = std::min(hist + 1, 3);
      eps_cur = eps_next;
      // with an empty basis the residual is only needed where it is tested:
      // after the last step of the batch (a non-finite value propagates to
      // it); with a basis every step needs the Newton correction, but only
      // the last one's residual is read
      if (c->p == 0) {
        if (b == batch - 1 && !eval(r)) return RPM_ERR_CUDA;
      } else if (!eval(r, b == batch - 1)) {
        return RPM_ERR_CUDA;
      }
    }
    trace(it, r);
    // stall: no halving of the residual in 3 (n_max + 1) steps -> re-centre
    if (r < 0.5 * r_best) {
      r_best = r;
      it_best = it;
    } else if (std::isfinite(r) && r > o.tol && it - it_best >= 3 * (o.n_max + 1) &&
               rebases < kMaxRebase) {
      if (!rebase() || !eval(r)) return RPM_ERR_CUDA;
      r_best = r;
      it_best = it;
    }
    if (std::isfinite(r) && r > o.tol && r <= o.diverge_factor * r0 && nu > o.n_max) {
      if (c->p < std::min(o.p_max, c->p_cap) && hist == 3) {
        const int p_before = c->p;
        want_rebase = false;
        if (!grow()) return RPM_ERR_CUDA;
        if (c->p != p_before && !eval(r)) return RPM_ERR_CUDA;
        if (want_rebase && rebases < kMaxRebase) {
          if (!rebase() || !eval(r)) return RPM_ERR_CUDA;
          r_best = r;
          it_best = it;
        }
      }
      nu = 0;
    }
  }

  if (c->p > 0 && (status == RPM_OK || status == RPM_ERR_NOT_CONVERGED)) {
    c->sb_p = c->p;   // what Z and W now hold, for a later solve of the same map
    c->sb_H = c->H;
    c->sb_key = key;
  }

  if (based) {   // eps = base + y
    ++c->launches;
    if (!ck(c, launch_axpby(base, 1.f, base, 1.f, eps_cur, c->n, c->st), "base")) return RPM_ERR_CUDA;
    eps_cur = base;
  }
  // outputs: eps, sigma = C : eps, <sigma>
  const size_t fb = c->fsz * sizeof(float);
  if (eps_out) {
    if (!ck(c, cudaMemcpyAsync(eps_out, eps_cur, fb,
                               out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st),
            "eps_out"))
      return RPM_ERR_CUDA;
  }
  float* sig_dev = sig_out ? (out_on_host ? D[0] : sig_out) : nullptr;
  if (sig_dev == eps_cur) sig_dev = D[1];
  c->launches += 2;
  if (!ck(c, launch_stress(c->g, eps_cur, sig_dev, c->partials, c->nblk, c->st), "stress") ||
      !ck(c, launch_reduce_partials(c->partials, c->nblk, 6, ds + kSums, c->st), "reduce"))
    return RPM_ERR_CUDA;
  if (sig_out && out_on_host) {
    if (!ck(c, cudaMemcpyAsync(sig_out, sig_dev, fb, cudaMemcpyDeviceToHost, c->st), "sig_out"))
      return RPM_ERR_CUDA;
  }
  if (!ck(c, cudaEventRecord(c->ev1, c->st), "event")) return RPM_ERR_CUDA;
  int kerr = 0;
  if (!ck(c, cudaMemcpyAsync(&kerr, c->g.err, sizeof(int), cudaMemcpyDeviceToHost, c->st),
          "error flag"))
    return RPM_ERR_CUDA;
  if (!ops.read_small(kSums, 6)) return RPM_ERR_CUDA;
  if (kerr) {
    c->err = "a kernel's bounded wait for an asynchronous copy gave up";
    cudaMemsetAsync(c->g.err, 0, sizeof(int), c->st);
    if (info) {
      inf.status = RPM_ERR_TIMEOUT;
      *info = inf;
    }
    return RPM_ERR_TIMEOUT;
  }
  for (int k = 0; k < 6; ++k) inf.mean_stress[k] = hs[kSums + k] / (double)c->n;
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  inf.ms = ms;
  for (size_t i = 0; i < c->prof_used; ++i) {
    float t = 0;
    if (cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) != cudaSuccess) continue;
    (c->prof_cat[i] == 0 ? inf.gamma_ms : inf.proj_ms) += t;
  }
  // sampled groups (opt.profile = k > 1) stand for all groups of their class
  if (c->prof_rec[0] > 0) inf.gamma_ms *= (float)((double)c->prof_seen[0] / (double)c->prof_rec[0]);
  if (c->prof_rec[1] > 0) inf.proj_ms *= (float)((double)c->prof_seen[1] / (double)c->prof_rec[1]);
  inf.launches = c->launches;
  inf.proj_bytes = c->proj_bytes;
  inf.iters = it;
  inf.gamma_applies = nF;
  inf.basis_size = c->p;
  inf.residual = r;
  inf.converged = status == RPM_OK;
  inf.status = status;
  if (info) *info = inf;
  if (status == RPM_ERR_NOT_CONVERGED) c->err = "max_iters reached";
  if (status == RPM_ERR_DIVERGED) c->err = "residual diverged";
  return status;
}

}  // namespace

extern "C" {

rpm_status rpm_solve(rpm_ctx* c, const double E[6], const float* eps0, float* eps_out,
                     float* sig_out, int out_on_host, rpm_solve_info* info) {
  if (!c || !E) return fail(c, RPM_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(E[k])) return fail(c, RPM_ERR_INVALID_ARG, "non-finite E");
  rpm_solve_info warm{};
  const float* start = eps0;
  float ms_warm = 0.f, gms_warm = 0.f, pms_warm = 0.f;
  long long launches_warm = 0;
  double pbytes_warm = 0.0;
  int f_warm = 0;
  if (c->opt.warm_tol > 0 && (!eps0 || c->opt.warm_from_eps0)) {
    // stage 1: Algorithm 3 (basis up to warm_p_max), C0 at the geometric mean of the phases
    double lmin = 1e300, lmax = 0, mmin = 1e300, mmax = 0;
    for (const auto& ph : c->phases) {
      lmin = std::min(lmin, ph.lambda);
      lmax = std::max(lmax, ph.lambda);
      mmin = std::min(mmin, ph.mu);
      mmax = std::max(mmax, ph.mu);
    }
    rpm_iso cw{c->opt.warm_c0_scale * std::sqrt(std::max(lmin, 0.0) * lmax),
               c->opt.warm_c0_scale * std::sqrt(std::max(mmin, 0.0) * mmax)};
    if (!(cw.mu > 0)) cw = c->c0;
    const rpm_options saved = c->opt;
    const rpm_iso c0_saved = c->c0;
    c->opt.scheme = RPM_SCHEME_POLARIZATION;
    c->opt.p_max = std::min(c->opt.warm_p_max, c->p_cap);
    c->opt.tol = c->opt.warm_tol;
    c->opt.max_iters = c->opt.warm_max_iters;
    float* stage = c->fields + 5 * c->fst;        // D[0]: free until the solve proper grows Z
    rpm_status s1 = ck(c, set_reference_medium(c, cw), "reference medium")
                        ? solve_impl(c, E, eps0, stage, nullptr, 0, &warm)
                        : RPM_ERR_CUDA;
    c->opt = saved;
    if (!ck(c, set_reference_medium(c, c0_saved), "reference medium")) return RPM_ERR_CUDA;
    if (s1 == RPM_ERR_CUDA || s1 == RPM_ERR_INVALID_ARG) return s1;
    if (s1 == RPM_OK || s1 == RPM_ERR_NOT_CONVERGED) {
      // a copy: the solve proper reuses D[0] as scratch
      float* warm_copy = c->fields + 6 * c->fst;
      if (!ck(c, cudaMemcpyAsync(warm_copy, stage, c->fsz * 4, cudaMemcpyDeviceToDevice, c->st),
              "warm copy"))
        return RPM_ERR_CUDA;
      start = warm_copy;
    }
    ms_warm = warm.ms;
    gms_warm = warm.gamma_ms;
    pms_warm = warm.proj_ms;
    launches_warm = warm.launches + 1;
    pbytes_warm = warm.proj_bytes;
    f_warm = warm.gamma_applies;
  }
  rpm_status s = solve_impl(c, E, start, eps_out, sig_out, out_on_host, info);
  if (s == RPM_ERR_CUDA) {
    cudaStreamSynchronize(c->st);
    if (info) info->status = s;
  }
  if (info && f_warm > 0) {
    info->warm_iters = warm.iters;
    info->warm_residual = warm.residual;
    info->ms += ms_warm;
    info->gamma_ms += gms_warm;
    info->proj_ms += pms_warm;
    info->launches += launches_warm;
    info->proj_bytes += pbytes_warm;
    info->gamma_applies += f_warm;
  }
  return s;
}

rpm_status rpm_effective_stiffness(rpm_ctx* c, double C_eff[36], rpm_solve_info info[6]) {
  if (!c || !C_eff) return fail(c, RPM_ERR_INVALID_ARG, "null argument");
  rpm_status worst = RPM_OK;
  for (int j = 0; j < 6; ++j) {
    double E[6] = {0, 0, 0, 0, 0, 0};
    E[j] = j < 3 ? 1.0 : 0.5;
    rpm_solve_info inf{};
    rpm_status s = rpm_solve(c, E, nullptr, nullptr, nullptr, 0, &inf);
    if (s == RPM_ERR_CUDA || s == RPM_ERR_INVALID_ARG) return s;
    if (s != RPM_OK && worst == RPM_OK) worst = s;
    for (int i = 0; i < 6; ++i) C_eff[i * 6 + j] = inf.mean_stress[i];
    if (info) info[j] = inf;
  }
  return worst;
}

}  // extern "C"

extern "C" {

rpm_status rpm_set_materials(rpm_ctx* c, int n_phases, const rpm_iso* phases, rpm_iso c0) {
  if (!c || !phases || n_phases < 1 || n_phases > 256)
    return fail(c, RPM_ERR_INVALID_ARG, "bad phases");
  if (!(c0.mu > 0) || !(c0.lambda + 2 * c0.mu > 0))
    return fail(c, RPM_ERR_INVALID_ARG, "bad reference medium");
  c->phases.assign(phases, phases + n_phases);
  c->g.n_phases = c->gb.n_phases = c->gp.n_phases = n_phases;
  ++c->mat_version;
  std::vector<float2> cm(256, make_float2(0.f, 0.f));
  for (int i = 0; i < n_phases; ++i)
    cm[i] = make_float2((float)phases[i].lambda, (float)phases[i].mu);
  if (!ck(c, cudaMemcpyAsync((void*)c->g.cmat, cm.data(), 256 * sizeof(float2),
                             cudaMemcpyHostToDevice, c->st),
          "materials") ||
      !ck(c, set_reference_medium(c, c0), "reference medium"))
    return RPM_ERR_CUDA;
  return RPM_OK;
}

rpm_status rpm_effective_stiffness_batch(const rpm_cell* cells, int n_cells, const rpm_options* opt,
                                         int n_workers, double* C_eff, rpm_solve_info* info,
                                         int* status) {
  if (!cells || n_cells < 0 || !C_eff || n_workers < 1) return RPM_ERR_INVALID_ARG;
  for (int i = 0; i < n_cells; ++i) {
    const rpm_cell& cl = cells[i];
    if (!cl.phase || !cl.phases || cl.n_phases < 1 || cl.n_phases > 256) return RPM_ERR_INVALID_ARG;
    if (!grid_supported(cl.grid.nx, cl.grid.ny, cl.grid.nz)) return RPM_ERR_UNSUPPORTED_GRID;
  }
  rpm_options o;
  rpm_default_options(&o);
  if (opt) o = *opt;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RPM_ERR_CUDA;
  // jobs: (cell, load); a worker keeps the cell's phase map and materials
  // loaded while it takes consecutive loads of the same cell.  With
  // share_basis a job is a whole cell, its six loads solved in turn on one
  // context so that each starts from the basis the previous one left.
  std::atomic<int> next{0};
  std::atomic<int> hard_error{RPM_OK};
  const int per_job = o.share_basis ? 6 : 1;
  const int n_jobs = 6 * n_cells / per_job;
  std::vector<int> cell_status(n_cells, RPM_OK);
  std::mutex status_mu;
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      hard_error = RPM_ERR_CUDA;
      return;
    }
    std::map<std::tuple<int, int, int>, rpm_ctx*> ctxs;   // contexts reused per grid shape
    int loaded_cell = -1;
    rpm_ctx* loaded_ctx = nullptr;
    for (;;) {
      const int job = next.fetch_add(1);
      if (job >= n_jobs || hard_error != RPM_OK) break;
      const int ci = job * per_job / 6;
      const rpm_cell& cl = cells[ci];
      const auto key = std::make_tuple(cl.grid.nx, cl.grid.ny, cl.grid.nz);
      rpm_ctx*& ctx = ctxs[key];
      if (!ctx) {
        if (rpm_create(&cl.grid, cl.phase, 0, cl.n_phases, cl.phases, cl.c0, &o, st, &ctx) != RPM_OK) {
          ctx = nullptr;
          hard_error = RPM_ERR_CUDA;
          break;
        }
        loaded_cell = ci;
        loaded_ctx = ctx;
      } else if (loaded_cell != ci || loaded_ctx != ctx) {
        if (rpm_set_phase(ctx, cl.phase, 0) != RPM_OK ||
            rpm_set_materials(ctx, cl.n_phases, cl.phases, cl.c0) != RPM_OK) {
          hard_error = RPM_ERR_CUDA;
          break;
        }
        loaded_cell = ci;
        loaded_ctx = ctx;
      }
      for (int j = job * per_job % 6; j < job * per_job % 6 + per_job; ++j) {
        double E[6] = {0, 0, 0, 0, 0, 0};
        E[j] = j < 3 ? 1.0 : 0.5;
        rpm_solve_info inf{};
        const rpm_status s = rpm_solve(ctx, E, nullptr, nullptr, nullptr, 0, &inf);
        if (s == RPM_ERR_CUDA || s == RPM_ERR_INVALID_ARG) {
          hard_error = s;
          break;
        }
        for (int i = 0; i < 6; ++i) C_eff[(size_t)ci * 36 + i * 6 + j] = inf.mean_stress[i];
        if (info) info[(size_t)ci * 6 + j] = inf;
        if (s != RPM_OK) {
          std::lock_guard<std::mutex> lk(status_mu);
          if (cell_status[ci] == RPM_OK) cell_status[ci] = s;
        }
      }
      if (hard_error != RPM_OK) break;
    }
    for (auto& kv : ctxs) rpm_destroy(kv.second);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  const int nw = std::max(1, std::min(n_workers, n_jobs));
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  if (status)
    for (int i = 0; i < n_cells; ++i) status[i] = cell_status[i];
  if (hard_error != RPM_OK) return (rpm_status)hard_error.load();
  for (int i = 0; i < n_cells; ++i)
    if (cell_status[i] != RPM_OK) return (rpm_status)cell_status[i];
  return RPM_OK;
}

}  // extern "C"
