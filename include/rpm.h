/*
 * rpm.h - C ABI of the GB300 RPM-FFT library.
 *
 * The library computes the strain and stress fields and the effective
 * stiffness of a periodic, voxelised, linear-elastic cell with isotropic
 * phases, by the fixed-point Lippmann-Schwinger scheme (Moulinec-Suquet,
 * Section 2 and Algorithm 1 of Peng, Nepal & Dayal, CMAME 2020) wrapped by
 * the recursive projection method (Section 3, Algorithm 2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A grid is nx * ny * nz voxels (x fastest), unit cell lengths lx, ly, lz.
 *   This build supports nx, ny in {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128,
 *   256} and nz in {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256};
 *   nz = 1 is a 2D plane-strain cell.  Other grids return
 *   RPM_ERR_UNSUPPORTED_GRID.
 * - A field is float32 [6][nz][ny][nx]: the symmetric tensor components
 *   11, 22, 33, 23, 13, 12 (tensor components, not engineering shears).
 *   Field pointers are DEVICE pointers unless an argument says otherwise,
 *   16-byte aligned, owned by the caller, and used in order on the stream
 *   given to rpm_create.
 * - A macroscopic strain E[6] is given in the same tensor components.
 * - The effective stiffness is a 6x6 Voigt matrix with engineering shear
 *   strains (row-major, order 11 22 33 23 13 12).
 * - Every call returns an rpm_status; on failure rpm_last_error() gives a
 *   message.  No call throws across the ABI.  A context is not thread-safe.
 */
#ifndef RPM_H
#define RPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rpm_ctx rpm_ctx;

typedef enum {
  RPM_OK = 0,
  RPM_ERR_INVALID_ARG = 1,      /* null pointer, bad size, bad option */
  RPM_ERR_UNSUPPORTED_GRID = 2, /* grid outside the supported set above */
  RPM_ERR_OOM = 3,              /* device allocation failed or exceeds the cap */
  RPM_ERR_CUDA = 4,             /* a CUDA call failed; see rpm_last_error */
  RPM_ERR_NOT_CONVERGED = 5,    /* max_iters reached above tolerance */
  RPM_ERR_DIVERGED = 6,         /* residual non-finite or grew past the bound */
  RPM_ERR_TIMEOUT = 7           /* reserved for bounded device waits */
} rpm_status;

typedef struct {
  int nx, ny, nz;
  double lx, ly, lz; /* cell lengths; 0 means 1 */
} rpm_grid;

/* Isotropic moduli: C_ijkl = lambda d_ij d_kl + mu (d_ik d_jl + d_il d_jk). */
typedef struct {
  double lambda, mu;
} rpm_iso;

/* Frequencies at index N/2 of an even axis (Nyquist) that coexist with another
 * non-zero frequency component get Gamma0 := 0; pure-axis Nyquist frequencies
 * are kept.  This keeps Gamma0_hat even in xi, hence the map real-valued.
 * It is the only mode of this build. */
enum { RPM_NYQ_ZERO_MIXED = 0 };

typedef struct {
  int n_max;             /* fixed-point steps between basis growths (Alg. 2), default 10 */
  int p_max;             /* cap on the unstable-basis size; 0 = basic scheme (Alg. 1); <= 256 */
  int max_iters;         /* fixed-point steps before RPM_ERR_NOT_CONVERGED, default 5000 */
  double tol;            /* stop when |F(eps) - eps| / (|E| sqrt(n)) <= tol, default 1e-6 */
  double t_ratio;        /* kappa: add one vector when |T22| <= kappa |T11| (Eq. 3.8), 0.1 */
  int nyquist;           /* RPM_NYQ_ZERO_MIXED (the only accepted value) */
  double diverge_factor; /* RPM_ERR_DIVERGED when residual > factor * initial, 1e10 */
  double max_device_gb;  /* refuse contexts needing more device memory; 0 = no cap */
  int profile;           /* k >= 1: time every k-th Gamma0 application and every k-th
                            projection group with CUDA events (1: all of them); 0: off */
  int scheme;            /* RPM_SCHEME_BASIC (Eq. 3.9, default) or RPM_SCHEME_POLARIZATION */
  double alpha, beta;    /* Algorithm 3 parameters (alpha = beta = 2: Accelerated scheme) */
  /* Warm start (cold start when warm_tol <= 0, the default): before the
   * solve proper, iterate Algorithm 3 (alpha, beta as above, no basis) with
   * the reference medium at the geometric mean (lambda_min lambda_max)^1/2,
   * (mu_min mu_max)^1/2 of the phases scaled by warm_c0_scale, until its own
   * increment is <= warm_tol (at most warm_max_iters steps); then run the
   * configured scheme from that strain to tol.  Only the stopping test of the
   * second stage decides convergence. */
  double warm_tol;
  double warm_c0_scale;  /* default 1 */
  int warm_max_iters;    /* default 2000 */
  int warm_p_max;        /* RPM basis of the warm-start stage (default 0: plain Algorithm 3) */
  int warm_from_eps0;    /* 0 (default): a caller eps0 replaces the warm-start stage;
                            1: the stage runs from eps0 (e.g. a learned guess) */
  int autotune;          /* 1: rpm_create times every available pair of plane-pass and
                            z-pass variants below on the context's grid and keeps the
                            fastest (rpm_set_options then keeps that choice while
                            autotune stays 1); 0 (default): the variants below */
  int plane_variant;     /* x/y passes: 0 (default) the fused plane kernels where the
                            grid has them (square planes 48-128), else as 1; 1 the
                            whole-plane kernels where the plane fits (nx = ny <= 128),
                            else as 2; 2 the five-pass row and y-pencil kernels */
  int pencil_variant;    /* z pass: 0 (default) the fused register-resident kernel where
                            the grid has it (nz 32, 48, 96, 128), else the default tile; 1 half,
                            2 twice the default pencils per block; 3 the default tile */
  int share_basis;       /* 1: a solve starts from the unstable basis (Z, W = F_u Z, H)
                            that an earlier solve of the same map left in the context --
                            F_u does not depend on the load E, so the six loads of
                            rpm_effective_stiffness share one basis (block RPM, same fixed
                            point); the basis is dropped when the phases, materials, C0,
                            scheme or Nyquist rule change.  Measured slower at p_max 20:
                            each unit load excites its own part of the slow eigenspace,
                            and a basis filled by the earlier loads cannot grow to take
                            it.  0 (default): every solve starts with an empty basis */
} rpm_options;

/* Fixed-point map wrapped by the solver.  BASIC: Eq. 3.9 (Algorithm 1).
 * POLARIZATION: Algorithm 3 (Section 5.5), read with s_b = alpha sigma -
 * beta C0:eps (the printed plus sign does not keep the solution a fixed
 * point); alpha = beta = 2 is the Accelerated scheme. */
enum { RPM_SCHEME_BASIC = 0, RPM_SCHEME_POLARIZATION = 1 };

typedef struct {
  int iters;           /* fixed-point steps taken */
  int gamma_applies;   /* applications of the Gamma0 map, including F_u z for H */
  int basis_size;      /* final size p of the unstable basis Z */
  int converged;       /* 1 if the residual met tol */
  int status;          /* rpm_status of the solve */
  double residual;     /* final fixed-point increment residual */
  double residual0;    /* residual of the initial guess */
  double mean_stress[6]; /* <sigma> of the returned strain field (FP64 sum) */
  float ms;            /* device time of the solve (CUDA events), milliseconds */
  float gamma_ms;      /* with opt.profile: device time of the Gamma0 applications (the
                          timed sample scaled to all of them) */
  float proj_ms;       /* with opt.profile: the same for the projection/combine kernels */
  long long launches;  /* CUDA kernels launched by the solve */
  double proj_bytes;   /* algorithmic bytes moved by the projection/combine kernels */
  int warm_iters;      /* steps of the warm-start stage (0: cold start) */
  double warm_residual;/* increment of the warm-start stage when it stopped */
  int basis_reused;    /* basis vectors taken over from an earlier solve (share_basis) */
} rpm_solve_info;

/* Fill `opt` with the defaults listed above. */
void rpm_default_options(rpm_options* opt);

/*
 * Create a context for one cell (Section 2: the periodic cell problem with
 * stiffness C(x) and reference medium C0, Eqs. 2.1-2.3).
 *   grid        grid and cell lengths.
 *   phase       uint8 phase id per voxel [nz][ny][nx], each < n_phases;
 *               a device pointer if phase_on_device, else a host pointer.
 *               Copied; the caller keeps ownership.
 *   phases      n_phases (1..256) isotropic moduli, host array, copied.
 *   c0          reference medium, lambda0 + 2 mu0 > 0, mu0 > 0.
 *   opt         options (may be NULL for defaults), copied.
 *   cuda_stream cudaStream_t for every later call (NULL: legacy stream).
 * The context owns its device buffers: the half spectrum, strain
 * iterates, the fixed-point history, the basis Z and F_u Z (p_max fields each).
 */
rpm_status rpm_create(const rpm_grid* grid, const uint8_t* phase, int phase_on_device,
                      int n_phases, const rpm_iso* phases, rpm_iso c0, const rpm_options* opt,
                      void* cuda_stream, rpm_ctx** out);

/* Replace the phase map (same grid); host or device pointer as flagged. */
rpm_status rpm_set_phase(rpm_ctx* ctx, const uint8_t* phase, int on_device);

/*
 * Record the residual history of later solves: residuals[k] is the
 * fixed-point increment residual after k fixed-point steps (k = 0: initial
 * guess) and basis_sizes[k] the basis size p then, for k < capacity.  While
 * the basis is empty the solver tests (and records) the residual only every
 * few steps; entries it skips are left untouched.  Host arrays owned by the
 * caller; either may be NULL; capacity 0 disables.
 */
rpm_status rpm_set_trace(rpm_ctx* ctx, double* residuals, int* basis_sizes, int capacity);

/* Replace the options (p_max may not exceed the value given at creation). */
rpm_status rpm_set_options(rpm_ctx* ctx, const rpm_options* opt);

enum {
  RPM_GAMMA_FULL_MAP = 0, /* out = F(in) = E - Gamma0 * ((C - C0) : in), Eq. 3.9, 2.4-2.5 */
  RPM_GAMMA_LINEAR = 1,   /* out = F_u in = -Gamma0 * ((C - C0) : in)  (E ignored) */
  RPM_GAMMA_RAW_TAU = 2,  /* out = -Gamma0 * in, `in` being a polarization tau (E ignored) */
  RPM_GAMMA_PROJECT = 3   /* out = E + Gamma0 * (C0 : in): the compatible strain field with
                             mean E nearest to `in` in the C0 energy (Sec. 2: Gamma0 C0 is
                             the projector onto compatible fluctuations); rpm_apply_gamma only */
};

/*
 * One application of the Lippmann-Schwinger fixed-point map (Eq. 3.9 in
 * polarization form; Eqs. 2.3-2.5): polarization, forward 3D real FFT,
 * Green operator of C0 per frequency (zero frequency set to E, mixed
 * Nyquist frequencies per opt.nyquist), inverse FFT.
 *   in, out  device fields [6][n]; may not alias.  E: host double[6].
 * Stream-ordered, asynchronous; uses the context's spectrum scratch.
 */
rpm_status rpm_apply_gamma(rpm_ctx* ctx, const float* in, const double E[6], float* out,
                           int flags);

/*
 * rpm_apply_gamma without a context and without any device allocation.
 * (The paper has no counterpart: this is a deployment variant of
 * rpm_apply_gamma.)
 *
 * For callers that cannot call cudaMalloc: an application that owns all
 * device memory through its own pool or plug-in allocator, or a loop that may
 * not pay cudaMalloc's implicit device synchronisation.  It computes exactly
 * what rpm_apply_gamma computes for the same grid, phases, C0, input, E and
 * flags, but its scratch (the half spectrum and the FFT/frequency/material
 * tables) is a set of fixed-size file-scope device arrays that every GPU
 * loading the library holds until the process exits (about 6.6 MB).
 *   grid     nx == ny <= 64 and nz <= 64 (and supported as above); other
 *            grids return RPM_ERR_UNSUPPORTED_GRID.
 *   phase    DEVICE pointer, uint8 [nz][ny][nx], ids < n_phases.
 *   phases   host array of n_phases (1..256) moduli; c0 the reference medium.
 *   in, out  device fields [6][n] (may not alias); E host double[6]
 *            (required for RPM_GAMMA_FULL_MAP); flags RPM_GAMMA_FULL_MAP,
 *            RPM_GAMMA_LINEAR or RPM_GAMMA_RAW_TAU (RPM_GAMMA_PROJECT needs a context).
 *   cuda_stream  stream for the copies and kernels (NULL: legacy stream).
 * The first call on a device looks up the arrays' device addresses (once per
 * device, safe from several host threads).  A call whose grid, phase moduli
 * and C0 differ from the previous call's on that device copies its tables
 * from host memory into the arrays (stream-ordered; from pageable memory the
 * runtime first waits for the stream's earlier work); a call with the same
 * ones copies nothing and only launches the kernels, asynchronously.  Never
 * call it on a stream that is being captured into a CUDA graph: such calls
 * are refused with RPM_ERR_INVALID_ARG.  All calls share the arrays, which
 * keep the last call's contents: calls whose kernels overlap on a GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Returns RPM_ERR_INVALID_ARG / RPM_ERR_UNSUPPORTED_GRID for bad arguments,
 * RPM_ERR_CUDA if a CUDA call fails.
 */
rpm_status rpm_apply_gamma_noalloc(const rpm_grid* grid, const uint8_t* phase, int n_phases,
                                   const rpm_iso* phases, rpm_iso c0, const float* in,
                                   const double E[6], float* out, int flags, void* cuda_stream);

/*
 * Solve the cell problem for macroscopic strain E (Algorithm 2; Algorithm 1
 * when p_max = 0).
 *   E          host double[6].
 *   eps0       optional device field, initial strain (NULL: eps0 = E).
 *   eps_out    optional output strain field; sig_out optional stress field.
 *   out_on_host  0: eps_out/sig_out are device pointers; 1: host pointers.
 *   info       optional; filled also on failure.
 * Float32 fields need two measures the paper's double-precision setting does
 * not: no basis growth from iterate differences below 1e-5 |xi| (the
 * rounding level of F), and re-centring, when such a growth is skipped or
 * the residual has not halved in 3 (n_max + 1) steps: the iterate is split
 * as eps = base + y and the iteration continues on y with the same linear
 * part and the defect F(base) - base (same fixed point; at most 16 times per
 * solve).
 * Synchronises the context stream before returning.
 */
rpm_status rpm_solve(rpm_ctx* ctx, const double E[6], const float* eps0, float* eps_out,
                     float* sig_out, int out_on_host, rpm_solve_info* info);

/*
 * Effective stiffness: six solves with the unit Voigt strains (shears as
 * engineering strain 1, i.e. eps_ij = eps_ji = 1/2); column j of C_eff is
 * <sigma> of load j.  C_eff: host double[36] row-major; info: optional
 * host array of 6.
 */
rpm_status rpm_effective_stiffness(rpm_ctx* ctx, double C_eff[36], rpm_solve_info info[6]);

/* Replace the phase moduli and the reference medium (same grid and phase map
 * semantics as rpm_create; the phase map itself is kept). */
rpm_status rpm_set_materials(rpm_ctx* ctx, int n_phases, const rpm_iso* phases, rpm_iso c0);

/* One cell of a batch: grid, host phase map [nz][ny][nx], host moduli, C0. */
typedef struct {
  rpm_grid grid;
  const uint8_t* phase;
  int n_phases;
  const rpm_iso* phases;
  rpm_iso c0;
} rpm_cell;

/*
 * Effective stiffness of many cells (grids may differ): the 6 x n_cells
 * solves (cell, unit load) are taken from a queue by n_workers host threads,
 * each with its own non-blocking CUDA stream and contexts reused per grid
 * shape, so solves of different cells and loads run concurrently on the
 * current device.  Each solve is the rpm_solve of `opt` (NULL: defaults).
 *   C_eff   host double[n_cells][36] (row-major 6x6 per cell, as
 *           rpm_effective_stiffness).
 *   info    optional host rpm_solve_info[n_cells][6].
 *   status  optional host int[n_cells]: RPM_OK or the first failure of the cell.
 * Returns RPM_OK if every solve converged, else the first failure (per-cell
 * detail in `status`); RPM_ERR_CUDA / RPM_ERR_INVALID_ARG abort the batch.
 * Blocks until all solves finished.
 */
rpm_status rpm_effective_stiffness_batch(const rpm_cell* cells, int n_cells, const rpm_options* opt,
                                         int n_workers, double* C_eff, rpm_solve_info* info,
                                         int* status);

/* Last error message of the context (never NULL). */
const char* rpm_last_error(const rpm_ctx* ctx);

/* Name of a status code. */
const char* rpm_status_string(rpm_status s);

/* Pencils per block of the z pass in use (the autotuner's choice when
 * options.autotune was set at creation); 0 for a null context. */
int rpm_pencil_tile(const rpm_ctx* ctx);

/* Plane-pass kernels in use: 0 fused, 1 whole-plane, 2 five-pass (the
 * autotuner's choice when options.autotune was set at creation); -1 for a
 * null context. */
int rpm_plane_variant(const rpm_ctx* ctx);

/* Self-check of the bounded waits (kernels that wait for an asynchronous
 * copy give up after about one second and report RPM_ERR_TIMEOUT instead of
 * hanging): runs one block on `cuda_stream` (NULL: the default stream) whose
 * barrier wait can never complete.  *gave_up = 1 when the wait gave up by
 * itself; *waited_ms = the kernel's duration (CUDA events).  Synchronizes
 * the stream.  Returns RPM_OK, or RPM_ERR_INVALID_ARG / RPM_ERR_CUDA. */
rpm_status rpm_bounded_wait_check(void* cuda_stream, int* gave_up, float* waited_ms);

/* Device bytes held by the context. */
size_t rpm_device_bytes(const rpm_ctx* ctx);

/* 1 if the grid is supported by this build, else 0. */
int rpm_grid_supported(int nx, int ny, int nz);

/* Release every resource of the context (NULL is allowed). */
void rpm_destroy(rpm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RPM_H */
