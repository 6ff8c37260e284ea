/*
 * splitsolve.h -- C ABI of the GB300 SplitSolve hot path (libsplitsolve.so).
 *
 * Problem (Eq. wf, Eq. negf): for each energy E and transverse momentum k,
 *   (E*S - H - Sigma_L (+) 0 (+) ... (+) Sigma_R) x = Inj
 * with H Hermitian and S positive definite, both block tridiagonal with n_b
 * diagonal blocks of size s_b.  The library computes
 *   - the lead self-energies Sigma_L, Sigma_R by surface-Green's-function
 *     doubling on the lead cells (decimation, Sec. 3A);
 *   - the first and last block columns Q of A^-1, A = E*S - H, by the block
 *     sweeps of Algorithm 1 and its mirror (Sec. 3B, SplitSolve preprocessing);
 *   - the 2*s_b boundary correction of Eq. x (Steps 1-4, Sherman-Morrison-
 *     Woodbury with Sigma^RB = B C): R = 1 - C Q, z = R^-1 C y, x = Q (b' + z);
 *   - the transmission T(E,k) = Re Tr[Gamma_L G_1n Gamma_R G_1n^H],
 *     Gamma = i (Sigma - Sigma^H).
 * Every step runs in CUDA kernels on the current device; there is no CPU
 * fallback: without a usable GPU every call returns SS_ERR_CUDA.
 *
 * Conventions
 *   - complex numbers are interleaved (re, im) float64 pairs (ss_c64);
 *   - every matrix block is s_b x s_b, row-major, contiguous;
 *   - arrays holding one entry per point are packed point after point in the
 *     order of the call's E/k_id arrays (points may have different s_b, n_b);
 *   - E, k_id, iters and status are HOST arrays; every other array argument
 *     is a device pointer when cfg.device_ptrs = 1 and a host pointer
 *     otherwise (host arrays are copied in/out inside the call);
 *   - all arrays are caller-owned; the library keeps no pointer to them
 *     after the call returns;
 *   - every call is enqueued on cfg.stream and synchronises that stream
 *     before returning (per-point status is reported on the host);
 *   - every call returns SS_OK (0) or one of the SS_ERR_* codes below and never
 *     aborts the process; ss_last_error() holds a one-line description.
 */
#ifndef SPLITSOLVE_H
#define SPLITSOLVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } ss_c64;
typedef struct ss_handle ss_handle;

/* status codes (return values and per-point status entries) */
#define SS_OK                0
#define SS_ERR_ARG           1  /* invalid argument (sizes, NULL, unknown k_id shape) */
#define SS_ERR_STATE         2  /* call order: e.g. no Hamiltonian for a k_id        */
#define SS_ERR_SINGULAR      3  /* zero or non-finite pivot in a block LU            */
#define SS_ERR_NOT_CONVERGED 4  /* decimation or refinement hit its iteration cap    */
#define SS_ERR_TIMEOUT       5  /* a bounded device wait expired                     */
#define SS_ERR_OOM           6  /* device workspace could not be allocated           */
#define SS_ERR_CUDA          7  /* CUDA runtime error (no device, launch failure)    */

/* precision modes */
#define SS_FP64          0  /* every step in FP64                                      */
#define SS_MIXED_BF16X3  1  /* large GEMMs on tcgen05 tensor cores, BF16 hi/lo split,
                               FP32 accumulation; FP64 panels, boundary, residual and
                               iterative refinement                                     */
#define SS_MIXED_BF16X6  2  /* as above with a 3-term BF16 split (6 products)          */
#define SS_MIXED_OZAKI   3  /* products on tcgen05 tensor cores from BF16 digit slices with
                               exact FP32 accumulation (FP64-accurate); FP64 panels,
                               pivoting, boundary solve and residual                     */

/* open-boundary (lead self-energy) methods */
#define SS_OBC_DECIMATION 0  /* Sancho-Rubio doubling of the surface Green's function   */
#define SS_OBC_FEAST      1  /* the leads' Bloch modes from a contour integral (Sec. 3A,
                                Eq. feast) with a Rayleigh-Ritz step, Sigma from them   */

typedef struct {
  int n_b_max;        /* largest n_b of any k_id (workspace sizing)                   */
  int s_b_max;        /* largest s_b of any k_id                                      */
  int max_points;     /* points processed together in one batch (workspace sizing)    */
  int max_inj;        /* largest n_inj passed to ss_solve                             */
  int precision;      /* SS_FP64 / SS_MIXED_*                                         */
  double eta;         /* lead broadening: z = E + i*eta inside the leads (default 1e-10) */
  double decim_tol;   /* doubling stops when max(|a|_1,|b|_1) <= decim_tol*|D|_1 (1e-14) */
  int decim_max_iter; /* doubling cap -> SS_ERR_NOT_CONVERGED (default 100)           */
  double ir_tol;      /* mixed: refinement target: backward error <= ir_tol (1e-14)   */
  int ir_max_iter;    /* mixed: refinement cap (default 10)                            */
  int warm_start;     /* 1: in ss_self_energy / ss_solve / ss_transmission / ss_dos,
                         seed the surface GF of each lead that has a network attached
                         (ss_set_warm_start) for points of the network's block size:
                         network seed, at most 8 steps of g <- (D - U g L)^-1, accepted
                         when the FP64 Dyson residual ||g (D - U g L) - 1||_F / sqrt(s_b)
                         is <= 1e-10, otherwise the plain doubling.  Default 0.       */
  void* stream;       /* cudaStream_t to enqueue on (NULL = legacy default stream)     */
  int device_ptrs;    /* 1: array arguments are device pointers                        */
  int use_graphs;     /* 1: replay decimation iterations from captured CUDA graphs     */
  int profile;        /* 1: time every kernel launch with CUDA events (eager launches,
                         no graphs); read the totals with ss_profile_read            */
  int partitions;     /* split every device into this many contiguous partitions whose
                         block sweeps run concurrently (Sec. 3B, Fig. pp), merged by one
                         Sherman-Morrison-Woodbury system of 2*partitions*s_b rows;
                         1..8, default 1 (SplitSolve's plain two-column split)        */
  int memory_lean;    /* 1: size the workspace for transmission-only calls
                         (ss_transmission, ss_solve with x = NULL), which keep only the
                         corner blocks of the inverse (running products) instead of both
                         block columns: (31 + 16 P + 4 P^2) s_b^2 complex per point
                         for P partitions (51 s_b^2 for one) instead of about
                         (2 n_b + 45) s_b^2 in FP64 with one partition.  Calls that
                         return wave functions or the density of states then fit fewer
                         points per batch, or fail with SS_ERR_OOM.  Default 0.        */
  int hermitian_sweeps; /* 1: factor the sweep blocks D_i = A_ii - A_{i,i+1} X_{i+1}
                         (Hermitian at real E) as L D L^H without pivoting, the
                         paper's no-pivoting Hermitian solver (Sec. 5E): only their
                         lower triangle is updated, half the factorisation work of
                         the pivoted LU.  A zero pivot gives SS_ERR_SINGULAR.
                         Default 0 (pivoted LU).                                      */
  int obc;            /* SS_OBC_DECIMATION (default) or SS_OBC_FEAST: the leads' modes
                         psi_q = lambda^q u of (L + lambda D + lambda^2 U) u = 0 (blocks of
                         z S - H at z = E + i*eta) inside the annulus 1/R < |lambda| < R,
                         from 2*feast_points contour solves (z B - A)^-1 B Y on |z| = R
                         and |z| = 1/R (one batched s_b x s_b LU each), an orthonormal
                         basis of the filtered subspace and a Rayleigh-Ritz step; the
                         modes going into the bulk (|lambda| < 1 right lead, > 1 left)
                         give F = U diag(lambda) U^+ and g = (D + U F)^-1 (right) or
                         (D + L F)^-1 (left), dropping modes outside the annulus (exact
                         when it holds all s_b of them).  Needs s_b <= 256 (subspace
                         up to 512).  Iteration counts are reported as 0.           */
  double feast_radius;/* R > 1 (default 50)                                               */
  int feast_points;   /* quadrature nodes per circle (default 16)                        */
  int feast_subspace; /* columns m0 of the random block Y (0 = 2 s_b, the full space)   */
  int tournament_pivoting; /* 1: the pivoted LU panels of up to 1024 rows choose their
                         pivots by a tournament over the 8 CTAs of a cluster (each CTA's
                         partial-pivoting candidates, then partial pivoting among them):
                         two cluster barriers per panel instead of one per column.
                         Another stable pivot order; results change at rounding level.
                         Default 0 (partial pivoting).                                */
  int lu_lookahead;     /* 1: in the two-level blocked LU the depth-nbo update of the
                         columns right of the next outer block runs on a second stream
                         while that block's panels are factored (row exchanges of those
                         columns wait for their block's far phase).  The same operations
                         in the same order on every element: results are bit-identical
                         to 0.  Default 0: the persistent exact GEMM holds every SM's
                         shared memory, so the panels cannot run beside it, and the
                         split update and extra exchange pass cost more than they hide. */
} ss_config;

/* Fill *cfg with the defaults listed above (n_b_max = 64, s_b_max = 512,
 * max_points = 8, max_inj = 64, SS_FP64, host pointers, graphs on, profiling off,
 * one partition, full workspace). */
void ss_config_default(ss_config* cfg);

/* Create a handle bound to the current CUDA device; allocates the device
 * workspace for cfg->max_points points of (n_b_max, s_b_max).
 * Errors: SS_ERR_ARG (NULL or non-positive sizes), SS_ERR_CUDA (no device),
 * SS_ERR_OOM (workspace does not fit). On error *h is set to NULL. */
int ss_create(ss_handle** h, const ss_config* cfg);

/* Store the blocks of H(k) and S(k) for momentum index k_id (0 <= k_id < 4096),
 * replacing any earlier ones.  H_diag, S_diag: n_b*s_b*s_b; H_upper, S_upper:
 * (n_b-1)*s_b*s_b, block i couples cell i to i+1; lower blocks are the
 * conjugate transposes.  lead_L / lead_R: NULL for a periodic copy of the end
 * cell (needs n_b >= 2), else 4*s_b*s_b holding {H00, H01, S00, S01} of the
 * lead, H01 coupling lead cell q to q+1 (the device-lead coupling is H01).
 * The data are copied into device memory owned by the handle.
 * Errors: SS_ERR_ARG (sizes above the handle's maxima, NULL blocks). */
int ss_set_hamiltonian(ss_handle* h, int k_id, int n_b, int s_b,
                       const ss_c64* H_diag, const ss_c64* H_upper,
                       const ss_c64* S_diag, const ss_c64* S_upper,
                       const ss_c64* lead_L, const ss_c64* lead_R);

/* Lead self-energies at real energies E[p] for the Hamiltonian k_id[p]:
 * Sigma_L = A_{1,0} g_L A_{0,1}, Sigma_R = A_{n,n+1} g_R A_{n+1,n} (A at real E,
 * surface Green's functions g at E + i*eta by doubling).  sigma_L/sigma_R
 * (optional, may be NULL): s_b*s_b per point.  iters (optional, host):
 * 2 per point (left, right doubling steps; -8 for a lead whose warm start was
 * accepted, cfg.warm_start).  status (optional, host): per
 * point SS_OK / SS_ERR_NOT_CONVERGED / SS_ERR_SINGULAR.  The results are
 * kept in the handle for later ss_solve / ss_transmission on the same
 * (E, k_id).  Returns the first non-OK point status, or a call-level error. */
int ss_self_energy(ss_handle* h, int n_pts, const double* E, const int* k_id,
                   ss_c64* sigma_L, ss_c64* sigma_R, int* iters, int* status);

/* Wave functions x = (A - Sigma)^-1 Inj for injections non-zero only in the
 * first and last block rows (Eq. wf; Steps 1-4 of Eq. x).  inj: per point
 * 2*s_b x n_inj row-major (rows of block 1, then rows of block n_b).
 * x: per point (n_b*s_b) x n_inj row-major; may be NULL, in which case only
 * G_1n is computed (and T cached for ss_transmission), keeping the corner
 * blocks of the inverse instead of its block columns (transmission-only mode).
 * 1 <= n_inj <= cfg.max_inj.  In the mixed modes x is refined in FP64 until
 * the normwise backward error ||Inj - (A - Sigma) x||_F /
 * (||A - Sigma||_F ||x||_F + ||Inj||_F) is <= ir_tol, until a correction no
 * longer halves the worst one of the batch, or until ir_max_iter
 * corrections; a point left above ir_tol gets SS_ERR_NOT_CONVERGED.  The transmission of each point is computed on the way and kept
 * for ss_transmission. */
int ss_solve(ss_handle* h, int n_pts, const double* E, const int* k_id,
             int n_inj, const ss_c64* inj, ss_c64* x, int* status);

/* Transmission T(E,k) = Re Tr[Gamma_L G_1n Gamma_R G_1n^H] per point (T:
 * n_pts doubles).  err_est (optional): FP64 path: |Im Tr| / max(1,|T|);
 * mixed path: the normwise backward error of the refined x (see ss_solve).  Reuses the
 * cached results of an immediately preceding ss_solve / ss_self_energy on the
 * same points; otherwise runs the whole pipeline. */
int ss_transmission(ss_handle* h, int n_pts, const double* E, const int* k_id,
                    double* T, double* err_est, int* status);

/* Local density of states per block of the open system:
 *   dos[p][i] = -Im Tr[G_ii] / pi,  G = (E S - H - Sigma_L (+) 0 (+) .. (+) Sigma_R)^-1,
 * for every block i = 1..n_b of point p (the retarded Green's function of
 * Eq. negf, whose diagonal gives the spectral weight the observables of
 * Sec. 2B are integrated from).  dos: n_b doubles per point, packed.
 * Computed by two block sweeps over A - Sigma (right- and left-connected
 * Schur complements of every block) and one LU per block of
 * (A_ii - Sigma^left_i - Sigma^right_i), Sigma from the doubling (cached when
 * the points equal the previous call's).  Needs 2 n_b s_b^2 complex of block
 * storage per point (ignores cfg.partitions).  status as in ss_self_energy,
 * SS_ERR_SINGULAR for a zero pivot in any block. */
int ss_dos(ss_handle* h, int n_pts, const double* E, const int* k_id, double* dos, int* status);

/* Release every device allocation of the handle (NULL is accepted). */
int ss_destroy(ss_handle* h);

/* One-line description of the last error on this handle ("" if none);
 * ss_last_error(NULL) describes the last ss_create failure. */
const char* ss_last_error(const ss_handle* h);

/* Number of kernel launches the library issued on this handle since
 * ss_create (graph replays count their kernel nodes). */
long long ss_launch_count(const ss_handle* h);

/* Host-side launch calls the pipeline calls (ss_self_energy, ss_solve,
 * ss_transmission, ss_dos) made on this handle since ss_create: one per eager
 * kernel launch or memset, one per CUDA-graph launch.  A plan whose launch
 * sequence repeats (same shapes and batch as before) is replayed from a graph
 * when cfg.use_graphs = 1. */
long long ss_host_launch_count(const ss_handle* h);

/* Complex GEMM with the library's kernels: C = op(A) op(B), op = identity or
 * conjugate transpose (transA / transB = 1), all DEVICE pointers, row-major
 * with leading dimensions lda, ldb, ldc (elements).  precision SS_FP64 runs
 * the FP64 kernel of the FP64 path; SS_MIXED_BF16X3 / X6 run the split-BF16
 * tcgen05 kernel (about 5e-6 relative error); SS_MIXED_OZAKI runs the
 * digit-sliced tcgen05 kernel (FP64-accurate).  Packing scratch is allocated
 * with cudaMallocAsync on `stream`.  The call synchronises `stream`.
 * Errors: SS_ERR_ARG, SS_ERR_OOM, SS_ERR_CUDA, SS_ERR_TIMEOUT (a bounded
 * pipeline wait inside the tensor-core kernel expired). */
int ss_zgemm(int precision, int m, int n, int k, const ss_c64* A, int lda, int transA, const ss_c64* B, int ldb,
             int transB, ss_c64* C, int ldc, void* stream);

/* The exact GEMM's split for inner dimension k (host only, no GPU needed):
 * slice width w (2k rounded up to 64), beta bits per digit, S digit slices,
 * and the exact FP32 passes: pass p accumulates the digit pairs
 * (t, pd[p] - t) for t = pt0[p] .. pt0[p] + pnp[p] - 1.  The arrays hold at
 * least 32 entries.  Returns SS_ERR_ARG when k < 1 or no exact split exists. */
int ss_exact_gemm_plan(int k, int* w, int* beta, int* S, int* npass, unsigned char* pd, unsigned char* pt0,
                       unsigned char* pnp);

/* Transmission from caller-provided blocks (the Caroli trace of the
 * transmission step): T[p] = Re Tr[Gamma_L G_1n Gamma_R G_1n^H] with
 * Gamma = i (Sigma - Sigma^H), for n_pts points of block size s_b.
 * sigma_L, sigma_R, G1n: DEVICE pointers, s_b*s_b complex per point, packed;
 * T: DEVICE pointer, n_pts doubles.  Scratch (4*s_b^2 + 1 complex per point)
 * is allocated with cudaMallocAsync on `stream` (a cudaStream_t, NULL = legacy
 * stream) and released before return; the call synchronises `stream`.
 * Errors: SS_ERR_ARG (sizes, NULL), SS_ERR_OOM, SS_ERR_CUDA; the message is
 * in ss_last_error(NULL). */
int ss_caroli_transmission(int n_pts, int s_b, const ss_c64* sigma_L, const ss_c64* sigma_R,
                           const ss_c64* G1n, double* T, void* stream);

/* Allocation-free variant of ss_caroli_transmission (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory, e.g.
 * code running under a pool allocator that owns the device, or a hook that
 * must not call cudaMalloc / cudaMallocAsync while another allocator is
 * active).  Same arguments and result as ss_caroli_transmission, but all
 * scratch comes from one fixed file-scope device array of about 4.6 MB that
 * every GPU loading the library holds until the process exits; the call
 * allocates nothing.  Limits: n_pts <= 256 and n_pts*s_b*s_b <= 65536,
 * larger problems are rejected with SS_ERR_ARG.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress).  The call
 * synchronises `stream` and uploads its descriptors from host memory, so it
 * cannot be captured into a CUDA graph: on a capturing stream it returns
 * SS_ERR_ARG without enqueuing anything.  Every call reuses the same array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  No part of the array needs to start at zero.
 * Errors: SS_ERR_ARG, SS_ERR_CUDA; the message is in ss_noalloc_last_error(),
 * which holds the text of the last failing call made by the CALLING thread. */
int ss_caroli_transmission_noalloc(int n_pts, int s_b, const ss_c64* sigma_L, const ss_c64* sigma_R,
                                   const ss_c64* G1n, double* T, void* stream);
const char* ss_noalloc_last_error(void);

/* Autotune the block LU-solve used by every sweep, doubling step and boundary
 * solve of blocks of size s_b: times a synthetic batch of n_problems
 * systems [D | B] (s_b x 3 s_b, the shape of the doubling and sweep
 * systems) for each panel width (8 and 16, or 32 above
 * s_b = 512) and, in SS_MIXED_OZAKI, each update arithmetic (0: FP64 SIMT,
 * 2: exact tensor-core products for the deep updates, 4: also for the outer
 * block's rows right of it, 3: for every update)
 * with one-level blocking or two-level blocking of outer width 32, 64, 128
 * or 256 (below s_b), and keeps the fastest
 * for this handle.  The factorisation is the block LU of Sec. 3B; the choice
 * changes the order of FP64 roundings only.
 * It also times the padded-work heuristic and the FP64 complex GEMM's five
 * tile shapes on a group of n_problems s_b x s_b x s_b products (FP64 path)
 * and, for the LU's wide rank-nb updates, on the whole LU solve of the chosen
 * blocking, and uses the fastest for those classes of products (-1 in the
 * cache: the heuristic).
 * cache_path (optional): a text file of lines "precision s_b n_problems nb
 * nbo upd ms" and "G precision s_b n_problems square_tile update_tile"; a
 * matching pair is reused without timing, a new result is appended.
 * Outputs (optional, host): chosen panel width nb, outer width nbo (0: one
 * level), update arithmetic upd, and its time in ms. */
int ss_autotune(ss_handle* h, int s_b, int n_problems, const char* cache_path, int* nb, int* nbo, int* upd,
                double* ms);

/* ------------------------------------------------------------------------
 * Learned warm start of the surface Green's function (not in the paper).
 * A 3-layer MLP maps features of (E, k) to the 2 s^2 real/imaginary entries
 * of one lead's surface Green's function (scaled by out_scale):
 *   features (n_in = 19): E, cos k, sin k, sin(m pi E), cos(m pi E), m = 1..8;
 *   layers n_in -> width -> width -> n_out, SiLU, mean-squared loss, Adam.
 * FP32 master weights, BF16 copies used by every GEMM, FP32 accumulation.
 * A tensor-core GEMM whose pipeline wait times out (2 s) sets a flag that the
 * next ss_mlp_get or ss_mlp_train_step with a loss reports as SS_ERR_CUDA.
 * All network arrays are DEVICE pointers, row-major, unless stated.
 * ------------------------------------------------------------------------ */
typedef struct ss_mlp ss_mlp;

/* Allocate a network for batches of up to max_batch rows; weights drawn from
 * U(-1/sqrt(fan_in), +1/sqrt(fan_in)) with a 64-bit LCG seeded by `seed`,
 * biases zero.  `stream` (cudaStream_t) orders every later call.
 * Errors: SS_ERR_ARG, SS_ERR_OOM, SS_ERR_CUDA. */
int ss_mlp_create(ss_mlp** net, int n_in, int width, int n_out, int max_batch, unsigned long long seed,
                  void* stream);
int ss_mlp_destroy(ss_mlp* net);
/* Replace the FP32 parameters W1 (width x n_in), b1, W2 (width x width), b2,
 * W3 (n_out x width), b3; params[6] are host (device_ptrs = 0) or device. */
int ss_mlp_set_params(ss_mlp* net, const float* const* params, int device_ptrs);
/* Copy the parameters (which = 0) or the last gradients (which = 1) to six
 * HOST arrays in the order above. */
int ss_mlp_get(ss_mlp* net, int which, float* const* out);
/* y (B x n_out, fp32) = network(x), x (B x n_in, fp32); y may be NULL (the
 * output stays in the network's buffer). */
int ss_mlp_forward(ss_mlp* net, int B, const float* x, float* y);
/* Forward, mean-squared loss against t (B x n_out), backward; with lr > 0
 * also one Adam step (beta1 0.9, beta2 0.999, eps 1e-8).  *loss (host, may
 * be NULL) receives the loss of this batch (the call then synchronises). */
int ss_mlp_train_step(ss_mlp* net, int B, const float* x, const float* t, float lr, double* loss);
/* GEMMs on the tcgen05 tensor cores (on = 1, the default when width and n_out
 * are multiples of 8) or on the tiled SIMT kernel (on = 0); both round the
 * same operands to BF16 and accumulate in FP32.  Errors: SS_ERR_ARG (on = 1
 * with a width or n_out that is not a multiple of 8). */
int ss_mlp_use_tensor_cores(ss_mlp* net, int on);
const char* ss_mlp_last_error(const ss_mlp* net);

/* Transverse momentum k of Hamiltonian k_id (default 0): the value the
 * warm-start network is fed for this k_id inside the pipeline
 * (cfg.warm_start).  Errors: SS_ERR_STATE (no Hamiltonian for k_id),
 * SS_ERR_ARG (non-finite k). */
int ss_set_momentum(ss_handle* h, int k_id, double k);

/* Attach a trained network as the warm start of lead `side` (0 left, 1 right)
 * for k-points with block size s_b = sqrt(n_out / 2); the network is not
 * owned.  out_scale: the factor the training targets were multiplied by. */
int ss_set_warm_start(ss_handle* h, ss_mlp* net, int side, double out_scale);

/* Surface Green's function g of lead `side` at E[p] + i*eta for the Hamiltonian
 * k_id[p] (s_b*s_b complex per point, packed; device or host per
 * cfg.device_ptrs).  kval[p] (host) is the transverse momentum fed to the
 * network.  With a warm start attached and use_warm = 1: g0 from the network,
 * then at most warm_iters steps of g <- (D - U g L)^-1 (right lead;
 * (D - L g U)^-1 left), accepted when ||g (D - U g L) - 1||_F / sqrt(s_b) <=
 * warm_tol; otherwise the plain doubling result is returned.  iters (host,
 * optional): fixed-point steps or doubling steps per point; seeded (host,
 * optional): 1 where the warm start was accepted. */
int ss_surface_gf(ss_handle* h, int n_pts, const double* E, const int* k_id, const double* kval, int side,
                  int use_warm, int warm_iters, double warm_tol, ss_c64* g, int* iters, int* seeded, int* status);

/* Kernel kinds for ss_profile_read. */
#define SS_KERNEL_ZGEMM      0  /* batched complex GEMM (all GEMM-shaped steps)      */
#define SS_KERNEL_FORM       1  /* elementwise forms / copies                         */
#define SS_KERNEL_LU_PANEL   2  /* LU panel factorisation                             */
#define SS_KERNEL_LU_ROW     3  /* LU row swaps + L11^-1 on the row block             */
#define SS_KERNEL_LU_BACK    4  /* backward substitution in a diagonal block of U     */
#define SS_KERNEL_NORM1      5  /* matrix 1-norms of the doubling test                */
#define SS_KERNEL_TRACE      6  /* transmission trace                                 */
#define SS_KERNEL_CHECK      7  /* doubling convergence flags                         */
#define SS_KERNEL_FILL       8  /* flag initialisation                                */
#define SS_KERNEL_TC_PACK_A  9  /* split-BF16 packing of A (3/6-product modes)        */
#define SS_KERNEL_TC_PACK_B 10  /* split-BF16 packing of B                            */
#define SS_KERNEL_TCGEMM    11  /* split-BF16 tcgen05 GEMM                            */
#define SS_KERNEL_ZGEMM32   12  /* (reserved: no FP32 GEMM is issued)                 */
#define SS_KERNEL_OZ_SCALE  13  /* row/column power-of-two scales of the exact GEMM   */
#define SS_KERNEL_OZ_PACK   14  /* BF16 digit slices of the exact GEMM                */
#define SS_KERNEL_OZGEMM    15  /* digit-sliced tcgen05 GEMM, exact FP32 accumulation */
#define SS_KERNEL_FROB2     16  /* Frobenius norms (warm-start judge, refinement)     */
#define SS_KERNEL_ZGEMM_LU  17  /* SS_KERNEL_ZGEMM launches issued by the block LU    */
#define SS_KERNEL_OZGEMM_LU 18  /* SS_KERNEL_OZGEMM launches issued by the block LU   */
#define SS_KERNEL_LU_HPANEL 19  /* Hermitian LDL^H panel (cfg.hermitian_sweeps)      */
#define SS_KERNEL_EIG       20  /* small dense eigenproblems (SS_OBC_FEAST)           */

/* With cfg.profile = 1: total device time (ms, CUDA events around each
 * launch on cfg.stream), algorithmic flops (GEMM kind only: 8 m n k per
 * complex product of every active problem, for every GEMM kind) and launch count of one kernel
 * kind since ss_create or the last ss_profile_reset.  Errors: SS_ERR_ARG. */
int ss_profile_read(ss_handle* h, int kind, double* total_ms, double* flops, long long* launches);
/* Flops the tensor pipe executed for kind SS_KERNEL_OZGEMM (2 * m * 2n *
 * digit pairs * padded slice width per product), for roofline fractions. */
int ss_profile_read_issued(ss_handle* h, int kind, double* issued_flops);
int ss_profile_reset(ss_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* SPLITSOLVE_H */
