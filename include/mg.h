/*
 * mg.h -- C ABI of the GB300 (sm_103a) adaptive multigrid solver for the
 * Wilson-Dirac equation D(U) psi = chi (Brannick, Brower, Clark, Osborn, Rebbi,
 * "Adaptive Multigrid Algorithm for Lattice QCD", arXiv:0707.4018).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice: d = 2, extents dims[0] = L0, dims[1] = L1, periodic in every
 *    direction; site index x = x0 + L0 * x1 (x0 fastest).
 *  - Gauge field U: complex128 (interleaved re, im) U[x][mu], mu = 0, 1; U_x^mu
 *    is the U(1) link from x to x + mu-hat (Nc = 1).
 *  - Fine spinor: complex128 psi[x][s], s = 0, 1 (two spin components).
 *  - Wilson operator (paper, definition following Eq. 1), with gamma_1 = sigma_1,
 *    gamma_2 = sigma_2 and the diagonal read as (d + m):
 *        (D psi)_x = (d + m) psi_x - 1/2 sum_mu [ (1 - gamma_mu) U_x^mu psi_{x+mu}
 *                                              + (1 + gamma_mu) U_{x-mu}^mu* psi_{x-mu} ]
 *  - Levels are numbered 0 (finest) .. levels-1 (coarsest). Level l+1 is the
 *    blocking of level l into blocks of block[l][0] x block[l][1] sites (the
 *    paper's geometric blocks S_j); coarse site j = block index
 *        j = (x0 / B0) + (L0 / B0) * (x1 / B1),
 *    in-block position s = (x0 % B0) + B0 * (x1 % B1).
 *  - A level-l vector is complex128 v[site][a], a < n_int(l), where n_int(0) = 2
 *    and n_int(l) = Nv[l-1] (the paper's intrinsic index s on coarse sites).
 *  - Coarse operator of level l >= 1 (paper, Eq. Galerkin, with A = D):
 *        y_j = sum_dir Y[j][dir] x_{j + offset(dir)},
 *    dir 0 = self, dir 1 = +0, 2 = -0, 3 = +1, 4 = -1 (source j + offset);
 *    exported row-major: Y[j][dir][row][col], complex128.
 *  - Near-null vectors / prolongator of level l: Nv[l] level-l vectors,
 *    exported as v[k][site][a]. The prolongator columns are the vectors cut to
 *    each block and block-orthonormalised (paper, Eq. P1 and the adaptive step).
 *
 * Memory and streams
 * ------------------
 *  All field pointers are DEVICE pointers on the current CUDA device unless a
 *  call says otherwise; the caller owns them. mg_setup copies U into library
 *  storage, so the caller may free U afterwards. A context owns its device
 *  workspace (allocated in mg_setup, freed in mg_destroy). Every call runs on
 *  the context's stream and returns after synchronising it.
 *
 * Errors
 * ------
 *  Every int-returning call returns MG_OK (0) or an mg_status code; a message
 *  is then available from mg_last_error() (thread-local). No C++ exception
 *  crosses this interface. On MG_ERR_NOT_CONVERGED, psi holds the last iterate
 *  and the stats are filled in.
 */
#ifndef MG_GB300_H
#define MG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 4

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* bad geometry, blocking, parameters or null pointer */
  MG_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  MG_ERR_OOM = 3,           /* device allocation failed */
  MG_ERR_NOT_CONVERGED = 4, /* max_iter reached before the tolerance */
  MG_ERR_NAN = 5,           /* a NaN/Inf or breakdown appeared in a reduction */
  MG_ERR_UNSUPPORTED = 6,   /* a valid request this build does not implement */
  MG_ERR_STATE = 7,         /* the hierarchy is incomplete for the request */
  MG_ERR_TIMEOUT = 8        /* a bounded device-side wait (grid barrier) ran out */
} mg_status;

typedef enum {
  MG_FP64 = 0, /* every level in FP64 */
  MG_FP32 = 1, /* FP64 outer flexible GCR; V-cycle (smoother, transfer, coarse ops) in FP32 */
  MG_FP16 = 2  /* half-precision storage with per-site FP32 norms, FP32 arithmetic. As a context
                  precision (d = 2): MG_FP32, except that the fine level of the solve's V-cycles
                  stores its links and the MR smoother's r and A r in half (12 bytes per site and
                  vector; the smoother's iterate, the cycle's input and the residual handed to the
                  restriction stay FP32); the setup runs as in MG_FP32. For mg_dslash: the half
                  layouts of mg_half_convert. */
} mg_precision;

typedef struct {
  int d;       /* number of dimensions: 2 (U(1)), or 4 (SU(3), where a call says so) */
  int dims[4]; /* lattice extents (dims[0] = L0, dims[1] = L1, ...) */
  int Nc;      /* colours: 1 (U(1), d = 2) or 3 (SU(3), d = 4) */
} mg_geom;

typedef struct {
  int levels;                       /* number of levels, 2..MG_MAX_LEVELS */
  int block[MG_MAX_LEVELS - 1][4];  /* block extents from level l to l+1 */
  int Nv[MG_MAX_LEVELS - 1];        /* near-null vectors kept on level l */
  int nu_pre, nu_post;              /* MR smoothing iterations before / after the coarse correction */
  double omega;                     /* MR under-relaxation (paper: 0.8) */
  int n_pass;                       /* adaptive setup passes (1 = relaxation only) */
  int nu_setup;                     /* MR iterations of the null-space relaxation (paper: Eq. relax) */
  int gcr_restart;                  /* outer flexible GCR restart length */
  int max_iter;                     /* outer iteration limit */
  int coarsest_lu_max;              /* coarsest dimension up to which a dense LU is used */
  double coarsest_tol;              /* relative residual of the iterative coarsest solve */
  int coarsest_restart;             /* restart length of the iterative coarsest solve (1..32) */
  int coarsest_max_iter;            /* iteration limit of the iterative coarsest solve */
  int precision;                    /* mg_precision */
  uint64_t seed;                    /* Philox4x32-10 key of the setup's random vectors */
  int max_rhs;                      /* right-hand sides one mg_solve_batch call may take (1..32) */
  int chiral_split;                 /* 1: split every fine near-null vector into its two chirality
                                       halves (1 +- gamma_5) / 2 before Gram-Schmidt, 2 Nv coarse dofs
                                       per site; required (and only built) for d = 4 */
} mg_params;

typedef struct {
  int iters;                         /* outer iterations */
  int converged;                     /* 1 if the true residual met the tolerance */
  double true_rel_residual;          /* |chi - D psi| / |chi|, recomputed in FP64 */
  long long level_apps[MG_MAX_LEVELS]; /* operator applications per level (level 0: fine D) */
  long long coarsest_iters;          /* iterations of the iterative coarsest solve */
  double ms;                         /* wall time of the call, stream-synchronised */
  int graphs;                        /* 1 if the V-cycles replayed a captured CUDA graph */
  double setup_s;                    /* seconds the context's setup took (mg_setup, mg_load_setup or
                                        mg_clone; host wall clock, stream-synchronised): the cost the
                                        paper amortises over right-hand sides and masses */
  double solve_s;                    /* seconds of this solve (ms / 1000) */
  long long fine_D_apps;             /* fine operator applications in this call: outer loop, true
                                        residuals and every V-cycle's smoothing and residual (the
                                        paper's cost measure); equals level_apps[0] */
} mg_stats;

typedef struct mg_ctx mg_ctx;

/* Defaults: 2 levels, 4x4 blocks, Nv = 8, MR 4 + 4 with omega = 0.8, 5 passes,
 * nu_setup = 8, GCR(16), max_iter 500, coarsest LU up to 2048, coarsest GCR
 * tol 1e-12 / restart 16 / 20000 iterations, FP64, seed 20070704, max_rhs 1. */
void mg_default_params(mg_params *p);

/*
 * Adaptive setup (paper: Eq. relax, Eq. P1, the adaptive passes and the
 * recursion to further levels; Eq. Galerkin for every coarse operator).
 *   ctx   out: new context (NULL on error)
 *   g     geometry (d = 2, Nc = 1 supported)
 *   U     device complex128 U[x][mu]; read during the call only
 *   m     mass (diagonal d + m)
 *   p     parameters (copied)
 *   stream  cudaStream_t to run on (NULL: the legacy default stream)
 * Random vectors: level-l vector k, complex dof i, is Philox4x32-10 with key
 * (seed lo, seed hi) and counter (i lo, i hi, k, l), followed by Box-Muller.
 * Errors: INVALID_ARG (extents not divisible by blocks, odd sizes, Nv larger
 * than a block's dofs, levels out of range), OOM, CUDA.
 */
int mg_setup(mg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, void *stream);

/* Solve D psi = chi to relative true residual tol by flexible GCR preconditioned
 * with one V-cycle per iteration (FP64 outer loop, true residual at restarts).
 * chi, psi: device complex128 [x][s] (d = 4: [x][s][c]); psi is overwritten (initial
 * guess 0). nrhs > 1 solves nrhs systems at the context mass with chi, psi holding
 * nrhs vectors back to back: the same as mg_solve_batch(ctx, nrhs, chi, psi, NULL, tol,
 * st) (the paper: many right-hand sides amortise one setup), so nrhs <= max_rhs.
 * st may be NULL, else nrhs entries. Returns NOT_CONVERGED (psi = last iterate)
 * after max_iter, INVALID_ARG for nrhs < 1. */
int mg_solve(mg_ctx *ctx, const void *chi, void *psi, int nrhs, double tol, mg_stats *st);

/* Solve nrhs systems D(m_v) psi_v = chi_v with one hierarchy (paper: many
 * right-hand sides amortise one setup; mass reuse, the setup at the lightest
 * mass serving heavier ones), in lockstep: every outer iteration applies one
 * batched V-cycle to all unfinished right-hand sides.
 *   nrhs  1..max_rhs of the setup parameters
 *   chi, psi  device complex128 [v][x][s], nrhs vectors back to back; psi is
 *         overwritten (initial guess 0)
 *   mass  host array of nrhs masses, or NULL for the context mass. Vector v
 *         sees every level's operator shifted by m_v - m: D(m_v) on the fine
 *         level and P^dagger D(m) P + (m_v - m) on the coarse ones, which is
 *         P^dagger D(m_v) P because the block-orthonormal P has P^dagger P = 1;
 *         the coarsest factors / preconditioners are prepared per mass
 *   st    NULL or nrhs entries: iters, converged and true_rel_residual per
 *         vector; level_apps, coarsest_iters, ms and graphs for the whole batch
 * A vector stops when its tracked residual meets tol and is confirmed by the
 * true residual at the next restart. Returns NOT_CONVERGED if any vector
 * missed tol within max_iter (outer iterations of the batch), INVALID_ARG for
 * nrhs outside 1..max_rhs or a non-finite mass.
 * d = 4 (the 4d SU(3) hierarchy): chi, psi complex128 [v][x][s][c]; every vector
 * solves at the context mass (mass NULL, else UNSUPPORTED); the batched
 * V-cycle's coarse solve is a lockstep GCR whose operator applications run on
 * tensor cores for all vectors at once (N = 48; BF16 operands, FP32 sums). */
int mg_solve_batch(mg_ctx *ctx, int nrhs, const void *chi, void *psi, const double *mass, double tol,
                   mg_stats *st);

/* nrhs[i] systems D_i psi = chi per context (2d contexts of any sizes, configurations and
 * masses; the paper: many gauge configurations, each with its own setup, and many right-hand
 * sides per setup), all solved by ONE launch of one CUDA graph: each context's outer flexible
 * GCR runs as a conditional WHILE node on the device (batched V-cycle, D apply, Gram-Schmidt
 * reduction, update and a control kernel that decides whether the loop goes on; the nrhs[i]
 * vectors of a context in lockstep, each stopping on its own residual), the loops of all
 * contexts side by side, with no host round trip per iteration. Gram-Schmidt is classical
 * with one pass; a restart starts a new basis from the recurrence residual. After the launch
 * the true residual b - D x of every system is recomputed in FP64; a system that misses tol
 * (rounding of the recurrence) is relaunched from its true residual.
 *   count      number of contexts (>= 1); every ctx[i] distinct, all on one device
 *   nrhs       NULL (one system each) or count entries in [1, max_rhs of the context]; all
 *              vectors of a context are solved at its mass
 *   chi, psi   arrays of device complex128 pointers, context i: nrhs[i] vectors [v][x][s]
 *              back to back (psi overwritten, initial guess 0)
 *   st         NULL or sum(nrhs) entries, context by context (ms / solve_s: the whole call)
 * Returns NOT_CONVERGED if any system missed tol within its max_iter, UNSUPPORTED for
 * d = 4 contexts. */
int mg_solve_multi(int count, mg_ctx *const *ctx, const int *nrhs, const void *const *chi, void *const *psi,
                   double tol, mg_stats *st);

/* Reuse the near-null vectors for another mass (paper: setup at the lightest
 * mass only, reused for heavier ones): rebuilds every Galerkin operator with
 * the kept prolongators and re-prepares the coarsest solve. */
int mg_update_mass(mg_ctx *ctx, double m);

/* A second context for another mass that reuses the setup of src (paper: the setup made
 * at the lightest mass serves the heavier ones): copies src's links and near-null vectors
 * / prolongators, builds every Galerkin operator at mass m and prepares the coarsest
 * solve, with no relaxation or adaptive pass. The result equals mg_update_mass(src, m)
 * applied to a copy of src; both contexts stay usable and independent (own stream,
 * own buffers), so solves at several masses can run concurrently.
 *   out     new context (NULL on error); free with mg_destroy
 *   stream  cudaStream_t the new context orders its work after
 * Errors: INVALID_ARG (null pointers), STATE (src has a stale level), UNSUPPORTED (d = 4),
 * OOM, CUDA. */
int mg_clone(mg_ctx *src, double m, void *stream, mg_ctx **out);

/* Adaptive setups of several gauge configurations (possibly of different lattice
 * sizes) at once (paper: one setup per configuration, amortised over its right-hand
 * sides and masses). Configuration i is set up exactly as mg_setup(&ctx[i], &g[i], U[i],
 * m[i], &p[i], stream) would, each on its own context stream and host thread, so the
 * setups run concurrently on the GPU; every context orders its work after `stream`.
 *   count  number of configurations (>= 1)
 *   ctx    out: count contexts (all NULL on error)
 *   g, U, m, p  arrays of count geometries, device link pointers, masses and parameters
 * The result of every configuration is the one mg_setup gives (bitwise). On any failure
 * every context made so far is destroyed and the first failure's status is returned. */
int mg_setup_batch(int count, mg_ctx **ctx, const mg_geom *g, const void *const *U, const double *m,
                   const mg_params *p, void *stream);

/* Write the context's adaptive setup to a file (paper: the near-null space found once is
 * reused for further masses and right-hand sides). The file holds the geometry, the
 * parameters, the mass, a 64-bit FNV-1a digest of the links the setup was made on, and
 * the near-null vectors of every level before orthonormalisation (complex128, the
 * mg_get_null_vectors layout), with a digest of that payload. The prolongators and
 * Galerkin operators are not stored: loading rebuilds them from the vectors.
 * Errors: INVALID_ARG (null pointers), STATE (a stale level), CUDA, and UNSUPPORTED when
 * the file cannot be written. */
int mg_save_setup(mg_ctx *ctx, const char *path);

/* A context from a saved setup: allocates as mg_setup does, copies U, then rebuilds every
 * level from the stored vectors (block Gram-Schmidt, Galerkin operator, coarsest-solve
 * preparation) without any relaxation or adaptive pass. The result, and every solve on
 * it, is bitwise equal to those of the context that was saved.
 *   U       device links of the same layout as mg_setup's; their digest must match the
 *           stored one (a setup belongs to its gauge field)
 *   stream  cudaStream_t the new context orders its work after
 * Errors: INVALID_ARG (null pointers, unreadable or corrupt file, version or size
 * mismatch, links whose digest differs), OOM, CUDA. */
int mg_load_setup(mg_ctx **ctx, const char *path, const void *U, void *stream);

/* The geometry, parameters and current mass of a context (any out-pointer may be NULL);
 * for a context from mg_load_setup these are the saved ones. */
int mg_context_info(const mg_ctx *ctx, mg_geom *g, mg_params *p, double *m);

/* Frees every device buffer of the context. NULL is a no-op. */
void mg_destroy(mg_ctx *ctx);

/* Message of the last failed call on this thread ("" if none). */
const char *mg_last_error(void);

/* ---- step-level entry points (one step of the hot path each) ------------- */

/* Fine Wilson operator out = D(U) in without a context (paper, definition of D).
 * precision MG_FP64: U, in, out complex128; MG_FP32: complex64; MG_FP16 (d = 2): the half
 * layouts of mg_half_convert. in and out must
 * not alias. stream: cudaStream_t. Asynchronous on the stream (no sync).
 * Geometries: d = 2 with Nc = 1 (layouts above), or d = 4 with Nc = 3: the
 * paper's four-dimensional SU(3) case (its outlook), in the DeGrand-Rossi basis
 *   gamma_1 = [[0,0,0,i],[0,0,i,0],[0,-i,0,0],[-i,0,0,0]], gamma_2 = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]],
 *   gamma_3 = [[0,0,i,0],[0,0,0,-i],[-i,0,0,0],[0,i,0,0]], gamma_4 = [[0,0,1,0],[0,0,0,1],[1,0,0,0],[0,1,0,0]],
 * site x = x0 + L0 (x1 + L1 (x2 + L2 x3)), psi[x][s][c] (s < 4, c < 3),
 * U[x][mu][a][b] (SU(3) link from x to x + mu-hat, row a, column b), diagonal 4 + m.
 * Errors: INVALID_ARG (extent < 2, volume >= 2^31, null or aliasing pointers,
 * unknown precision), UNSUPPORTED (other d / Nc). */
int mg_dslash(const mg_geom *g, const void *U, double m, const void *in, void *out, int precision, void *stream);

/* Half-precision storage of 2d fields (the FP16 storage of the mixed-precision scheme): a spinor
 * field of nsites sites is [nsites][2] IEEE half pairs (re, im), scaled by a per-site FP32 norm
 * (the site's largest |Re| or |Im|), followed by [nsites] float norms: 12 bytes per site, value =
 * norm x half. Links are [nsites][2] half pairs (cos, sin), unscaled (|U| = 1): 8 bytes per site.
 * mg_dslash with MG_FP16 takes U, in and out in these layouts (FP32 arithmetic; the output is
 * rescaled by its own per-site norm before it is rounded). Conversions:
 *   what 0: complex spinor (precision MG_FP64 / MG_FP32, [x][s]) -> half spinor
 *   what 1: half spinor -> complex spinor
 *   what 2: complex links [x][mu] -> half links
 * Asynchronous on stream. Errors: INVALID_ARG (null or aliasing pointers, bad what / precision). */
int mg_half_convert(int what, int precision, const void *in, void *out, long long nsites, void *stream);

/* Apply the level-l operator (l = 0: D; l >= 1: the Galerkin stencil) in FP64. */
int mg_level_apply(mg_ctx *ctx, int level, const void *in, void *out);

/* Restriction r_c = P_l^dagger r (level l -> l+1) and prolongation f = P_l e_c,
 * FP64, level vectors in the canonical layouts above. */
int mg_restrict(mg_ctx *ctx, int level, const void *fine, void *coarse);
int mg_prolong(mg_ctx *ctx, int level, const void *coarse, void *fine);

/* One V-cycle x = V b on the finest level in the context's precision
 * (paper: the five V-cycle steps). b, x: device complex128 [x][s]. */
int mg_vcycle(mg_ctx *ctx, const void *b, void *x);

/* One coarsest-level solve x = A_c^{-1} b (paper: the coarsest level of the
 * V-cycle is an exact solve), FP64, coarsest-level layout [site][a]: dense LU
 * when the coarsest dimension is <= coarsest_lu_max, else the persistent GCR
 * kernel to relative residual coarsest_tol. iters (may be NULL): iterations of
 * the iterative solve (0 for LU). ms (may be NULL): device time of the solve,
 * from CUDA events recorded on the context's stream around it. */
int mg_coarsest_solve(mg_ctx *ctx, const void *b, void *x, long long *iters, double *ms);

/* nu MR iterations x = R b from x = 0 on level l (FP64), omega from the params. */
int mg_smooth(mg_ctx *ctx, int level, const void *b, void *x, int nu);

/* Replace the near-null vectors of level l by Nv[l] caller vectors (device,
 * complex128 [k][site][a]), then block-orthonormalise them into P_l and
 * rebuild the Galerkin operator of level l+1 (and the coarsest solve if l+1 is
 * the coarsest). Levels below l+1 become stale until rebuilt (MG_ERR_STATE
 * from calls that need them). */
int mg_build_level(mg_ctx *ctx, int level, const void *vectors);

/* Export level data (device destination buffers, complex128):
 *   mg_get_null_vectors: the Nv[l] near-null vectors of level l (before orthonormalisation)
 *   mg_get_prolongator:  the block-orthonormal columns of P_l as Nv[l] level vectors
 *   mg_get_coarse_op:    Y of level l >= 1, [j][dir][row][col]
 * and sizes: n_sites(l), n_int(l). */
int mg_get_null_vectors(mg_ctx *ctx, int level, void *out);
int mg_get_prolongator(mg_ctx *ctx, int level, void *out);
int mg_get_coarse_op(mg_ctx *ctx, int level, void *out);
int mg_level_size(mg_ctx *ctx, int level, long long *n_sites, int *n_int);

/* Fine-level MR smoother that allocates nothing: x = nu MR iterations (omega) for
 * D(U) x = b from x = 0, the same computation as mg_smooth at level 0, for callers
 * that cannot allocate device memory when they smooth (inside a stream capture, or
 * under a framework that owns the whole memory pool). The paper has no counterpart;
 * this is a library convenience.
 *   g: d = 2, Nc = 1, at most 65536 sites (256 x 256); larger lattices are rejected
 *      with MG_ERR_INVALID_ARG before any device work.
 *   U, b, x: device complex128 ([x][mu], [x][s], [x][s]) on the CURRENT device (the
 *      scratch array is per device); b and x must not alias. x on another device, or not
 *      device memory, is rejected with MG_ERR_INVALID_ARG.
 *   stream: cudaStream_t of the current device; the call is asynchronous on it.
 * Scratch lives in one fixed device array (about 4 MB, held on every GPU that
 * loads the library until exit), shared by all calls on a device; calls whose
 * work overlaps on the GPU race on it. The first call on a device looks up the
 * array's device address; make that first call before any stream capture. */
int mg_smooth_fine_noalloc(const mg_geom *g, const void *U, double m, const void *b, void *x, int nu, double omega,
                           void *stream);

/* Coarse stencil apply on tensor cores for many right-hand sides (paper: the coarse
 * operator P^dagger D P of Eq. Galerkin applied to a block of vectors, the contraction of
 * multi-RHS solves): out_n = A_l in_n for n < nrhs.
 *   d = 2: level 1..levels-1 with N = 8 dofs per coarse site. Per site and direction the
 *          complex 8 x 8 block is the real 16 x 16 matrix [[Re, -Im], [Im, Re]], applied with
 *          mma.sync m16n8k16; the tile shape is chosen by the autotuner (mg_autotune_report).
 *          Needs a context set up with precision MG_FP32 (its FP32 operator is rounded to BF16).
 *   d = 4: level 1 with N = 48 (Nv = 24): the 48 x 48 complex block is the real 96 x 96
 *          matrix [[A, -B], [B, A]] (A = Re Y, B = Im Y), applied as 16 x 16 tiles of A and
 *          B (-B by a sign flip): 108 mma.sync per warp of 16 rows x 8 vectors; the FP64
 *          operator is rounded to BF16 (either precision).
 *   in, out  device complex64 [n][site][dof], nrhs level vectors back to back (caller-owned)
 * tensor_cores = 1: operands rounded to BF16, products summed in FP32 (relative error about
 * 2^-8 of sum |Y| |x|). d = 4 only: 2 splits every vector entry into BF16 hi + lo (twice the
 * MMAs; the error is then the operator's rounding), 3 splits the operator as well and sums
 * hi hi + hi lo + lo hi (three times the MMAs, twice the operator bytes; about 2^-16 of
 * sum |Y| |x|). tensor_cores = 0 runs the same product on CUDA cores in FP32 (the comparison
 * path). Errors: INVALID_ARG (level, nrhs < 1, null pointers, tensor_cores outside 0..3,
 * overlapping in and out), UNSUPPORTED (d = 2 with an FP64 context, N != 8 or
 * tensor_cores > 1; d = 4 with N != 48). */
int mg_coarse_apply_mrhs(mg_ctx *ctx, int level, int nrhs, const void *in, void *out, int tensor_cores);

/* ---- learned near-null setup --------------------------------------------------------
 * The paper finds the near-null vectors by relaxation on the homogeneous problem
 * (Eq. relax) refined by the adaptive passes, and notes that this setup is the cost to be
 * amortised. The learned setup predicts them instead with a gauge-covariant network and
 * keeps the plain setup as its fallback and its judge (the measured MG convergence rate).
 *
 * Network: 4 parallel-transport convolution layers, cin -> channels -> channels ->
 * channels -> nv (each channel a 2-spin field); per site x and channel-spin index
 * l = 2 c + s,
 *     a_x = sum_dir W_dir T_dir(h)_x,  dir = self, +0, -0, +1, -1,
 *     T_self h_x = h_x,  T_{+mu} h_x = U_x^mu h_{x+mu},  T_{-mu} h_x = conj(U_{x-mu}^mu) h_{x-mu};
 * hidden layers h = a / sqrt(1 + |a_c|^2) per channel c (both spins), the last layer is
 * linear and its channel k is the predicted vector v_k. The weights W_dir[l_out][l_in]
 * (complex, FP32) act on channel and spin only, so the network commutes with gauge
 * transformations. Activations are stored in bfloat16, arithmetic is FP32. The input is
 * cin complex Gaussian fields: channel c, dof (x, s) is the setup's Philox4x32-10 draw
 * with key noise_seed, counter (2 x + s, 0, c, 0x4E4E), Box-Muller as in mg_setup.
 * Loss (rotation invariant, per block b of the blocking, rows (site in block, spin)):
 *     L_b = sum_k |(1 - Q_b Q_b^dagger) V_b e_k|^2,  loss = mean_b L_b / nv in [0, 1],
 * Q_b an orthonormal basis of the predicted vectors on b, V_b the target block-orthonormal
 * prolongator columns (mg_get_prolongator of a plain setup).
 * Weights are exchanged as complex64, layers packed [l][5][2 co][2 ci]. */
typedef struct mg_nullnet mg_nullnet;

/* New network with weights drawn from a seeded Gaussian (variance 1 / (10 ci) per
 * component). cin, channels in [1, 16], nv in [1, 8]. */
int mg_nullnet_create(mg_nullnet **net, int cin, int channels, int nv, uint64_t seed);
void mg_nullnet_destroy(mg_nullnet *net);
long long mg_nullnet_weight_count(const mg_nullnet *net); /* complex weights, all layers */
int mg_nullnet_get_weights(mg_nullnet *net, void *host_out);  /* complex64 [count] */
int mg_nullnet_set_weights(mg_nullnet *net, const void *host_in); /* resets the Adam state */

/* Forward pass on nfields fields of geometry g (d = 2, Nc = 1): U device complex128
 * [f][x][mu]; noise_seeds host [nfields]; out device complex64 [f][x][2 nv] (channel k,
 * spin s at 2 k + s). Synchronous. */
int mg_nullnet_forward(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const uint64_t *noise_seeds,
                       void *out, void *stream);

/* Loss and its conjugate cogradient dloss/dW^* (host complex64 [count], may be NULL) for
 * nfields fields against targets (device complex128 [f][k][x][s], block-orthonormal on the
 * blocks block[0] x block[1], at most 16 sites). The real-parameter gradient is 2 (Re, Im). */
int mg_nullnet_gradient(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const uint64_t *noise_seeds,
                        const void *target, const int *block, double *loss, void *grad, void *stream);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on batches of `batch`
 * fields taken cyclically from the nfields (U, target as for mg_nullnet_gradient), each
 * draw with fresh noise (seed + (draw << 20)). losses: host [steps] or NULL. */
int mg_nullnet_train(mg_nullnet *net, const mg_geom *g, int nfields, const void *U, const void *target,
                     const int *block, int steps, int batch, double lr, uint64_t seed, double *losses,
                     void *stream);

/* Setup with learned near-null vectors (d = 2): the network predicts the level-0 vectors
 * from noise_seed (it needs nv == p->Nv[0]) in place of the random start and relaxation of
 * the first pass (Eq. relax); nu_refine MR iterations on D v = 0 refine them (0: none), then
 * block Gram-Schmidt and the Galerkin operator build level 1. Passes 2..p->n_pass follow as
 * in the plain setup (p->n_pass = 1: none), and deeper levels get the plain adaptive setup
 * after each pass. The judge: the asymptotic convergence factor of the
 * V-cycle iteration e <- (1 - V D) e on a random vector over rate_steps steps (as
 * mg_convergence_rate). If it exceeds max_rate, the plain adaptive setup replaces the
 * learned one (the fallback) and *used_learned is 0. rate (may be NULL): the factor of the
 * hierarchy kept. stats of later solves report the whole call's time as setup_s. */
int mg_setup_learned(mg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, mg_nullnet *net,
                     uint64_t noise_seed, int nu_refine, double max_rate, int rate_steps, int *used_learned,
                     double *rate, void *stream);

/* Asymptotic convergence factor of the multigrid iteration: e_0 a Philox Gaussian vector
 * (seed), e_{i+1} = e_i - V(D e_i) with the context's V-cycle, rate = (|e_steps| / |e_1|)^(1
 * / (steps - 1)) (steps >= 2). d = 2. */
int mg_convergence_rate(mg_ctx *ctx, int steps, uint64_t seed, double *rate);

/*
 * MG-preconditioned conjugate gradients on the normal equations: the paper's own experiment
 * (numerical-results section; Eq. vcycle in its hermitian form). The operator is A = D^dagger D;
 * the hierarchy is built by the adaptive procedure on A (Eq. relax with nu_setup MR steps on
 * A x = 0 from Philox vectors, block Gram-Schmidt, n_pass - 1 adaptive passes v <- v - V(A v),
 * level by level); the coarse operators P^dagger A P are 9-point stencils (D^dagger D reaches the
 * diagonal neighbours); every non-coarsest level relaxes with the degree-2 MR polynomial whose
 * coefficients come from two MR steps (omega) on a fixed Philox vector and are then held fixed, so
 * R = R^dagger and the V-cycle is hermitian; the coarsest level is solved by dense LU (at most 4096
 * dofs). All arithmetic is FP64.
 *   mg_cg_setup: g (d = 2, Nc = 1), U device complex128 [x][mu] (copied), mass m, parameters p
 *     (levels, block, Nv, n_pass, nu_setup, omega and seed are used; blocks at least 2 x 2, and
 *     every coarse extent at least 3). Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA, NAN.
 *   mg_cg_solve: psi = D^{-1} chi through A psi = D^dagger chi by CG from psi = 0, preconditioned
 *     by one V-cycle per iteration when `precondition` is nonzero (plain CG otherwise), until the
 *     recursive residual is at most tol |D^dagger chi| or after max_iter iterations. chi, psi:
 *     device complex128 [x][s]. st (may be NULL): iterations, the recomputed relative residual of
 *     the normal equations, and the fine A applications of the call (the paper's cost measure: 6
 *     per MG-CG iteration, 1 per CG iteration). NOT_CONVERGED leaves the last iterate in psi.
 *   mg_cg_get_coarse_op: the level-l (l >= 1) stencil Y[j][o][row][col] (o = 3 (o1 + 1) + (o0 + 1)
 *     for the neighbour j + o), device complex128, nsites x 9 x N x N.
 */
typedef struct mg_cg_ctx mg_cg_ctx;
typedef struct {
  int iters;              /* CG iterations */
  int converged;          /* 1 if the recursive CG residual met the tolerance (the paper's criterion) */
  double rel_residual;    /* |D^dagger chi - A psi| / |D^dagger chi|, recomputed in FP64 afterwards */
  long long fine_apps;    /* fine A = D^dagger D applications of the iterations */
  double ms;              /* wall time of the call, stream-synchronised */
} mg_cg_stats;
int mg_cg_setup(mg_cg_ctx **ctx, const mg_geom *g, const void *U, double m, const mg_params *p, void *stream);
int mg_cg_solve(mg_cg_ctx *ctx, const void *chi, void *psi, double tol, int max_iter, int precondition,
                mg_cg_stats *st);
int mg_cg_get_coarse_op(mg_cg_ctx *ctx, int level, void *out);
int mg_cg_destroy(mg_cg_ctx *ctx);

/* Launch shapes picked by the library's autotuner so far (the tensor-core coarse apply
 * times its six tile shapes -- warps per CTA x vector tiles per warp -- on first use for
 * each lattice and vector count, and keeps the fastest; all shapes give bitwise the same
 * result). Writes "key=variant;..." into buf (NUL-terminated, truncated to len - 1
 * characters) and returns the full length. buf may be NULL when len is 0. */
size_t mg_autotune_report(char *buf, size_t len);

/* Self-test of the bounded device-side wait used by the persistent kernels (a
 * failure-detection check; the paper has no counterpart). Launches a 2-CTA
 * cooperative kernel whose grid barrier expects 2 + missing_arrivals arrivals
 * (missing_arrivals 0 or 1). With 1, nothing ever releases the barrier: each
 * wait gives up after a bounded number of polls (milliseconds), the kernel
 * returns and the call reports MG_ERR_TIMEOUT; the context stays usable.
 * With 0 the barrier completes and the call returns MG_OK. */
int mg_selftest_barrier(int missing_arrivals, void *stream);

/* Measured fused-multiply-add throughput of the current GPU in TFLOP/s (2 flops per FMA),
 * precision MG_FP64 or MG_FP32: a grid of 8 CTAs per SM, each thread running 8 independent
 * FMA chains, timed with CUDA events on `stream` after a warm-up launch. The roofline
 * denominator of the ALU-bound kernels (the paper has no counterpart; a measurement aid). */
int mg_alu_peak(int precision, double *tflops, void *stream);

/* Number of kernels this library has launched since the process started. */
long long mg_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_GB300_H */
