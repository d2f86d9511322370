/*
 * lqcd.h -- C ABI of the GB300 multi-rhs Wilson(-clover) Dirac operator and batched GMRES.
 *
 * Every function returns an lqcd_status (0 = OK, > 0 warning, < 0 error) and never
 * throws or aborts; lqcd_last_error() gives a thread-local message for the last
 * failing call on the calling thread. All GPU work is enqueued on the caller's
 * CUDA stream (`stream` is a cudaStream_t passed as void*, NULL = legacy default
 * stream); no call synchronises the device except where stated.
 *
 * Conventions (the paper's Sec. III-A-1 with the readings stated here):
 *   dims = {T, Z, Y, X}, every extent even and >= 2; direction mu = 0, 1, 2, 3 is
 *   t, z, y, x. Site number ((t*Z + z)*Y + y)*X + x (last coordinate fastest).
 *   V = T*Z*Y*X sites, V/2 per parity; parity of a site = (t+z+y+x) mod 2,
 *   even = 0. Fermion boundary condition in time is `time_bc` (+1 periodic,
 *   -1 antiperiodic), space is periodic.
 *   Gamma matrices in the chiral basis gamma_mu = [[0, P_mu], [P_mu^dag, 0]],
 *   P_t = 1, P_k = i sigma_k; gamma5 = diag(-1, -1, +1, +1).
 *   D psi(x) = A(x) psi(x) - sum_mu [ pi^-_mu (x) U_mu(x) psi(x+mu)
 *                                     + pi^+_mu (x) U_mu(x-mu)^dag psi(x-mu) ],
 *   pi^+-_mu = (1 +- gamma_mu)/2, A(x) = (4 + m0) 1 - C(x),
 *   C(x) = (c_sw/32) sum_{mu,nu} gamma_mu gamma_nu (x) (Q_mu,nu(x) - Q_nu,mu(x))
 *   (clover-leaf sum Q of the four plaquettes in the mu-nu plane at x).
 *   Odd-even (Sec. III-A-2): the Schur complement on the odd sites,
 *   S = A_oo - D_oe A_ee^{-1} D_eo.
 *
 * Canonical ("user") layouts, complex numbers stored interleaved (re, im):
 *   gauge field: complex128 [V][4][3][3], U[x][mu][row][col] (row-major 3x3).
 *   spinor block: complex [nrhs][n_sites][4][3] (spin, colour), rhs outermost;
 *   n_sites = V for full-lattice vectors, V/2 for one parity (its sites in
 *   increasing site number).
 * Packed ("internal") layout: complex [n_sites/S][12][S][nrhs] with component
 * index 3*spin + colour and the rhs index innermost (Eq. (2)'s rows stored
 * rhs-fastest), S = lqcd_site_tile(ctx, nrhs). Full-lattice packed vectors hold the
 * even sites first, then the odd sites, each in increasing site number. The
 * packed layout is what the operator kernels read and write; its byte size is
 * lqcd_packed_bytes().
 *
 * Pointers: unless a parameter says "host or device", pointers are device
 * pointers that stay owned by the caller. The library owns its copies of the
 * gauge field, the clover blocks and all workspace, and frees them in
 * lqcd_free(). Device pointers must be 16-byte aligned.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int lqcd_status;
enum {
  LQCD_OK = 0,
  LQCD_NOT_CONVERGED = 1,   /* warning: solve stopped at max_restarts; x holds the last iterate */
  LQCD_ERR_ARG = -1,        /* invalid argument (null pointer, bad size, odd extent, ...) */
  LQCD_ERR_OOM = -2,        /* device or pinned-host allocation failed */
  LQCD_ERR_CUDA = -3,       /* a CUDA runtime call failed; lqcd_last_error() has its text */
  LQCD_ERR_NONFINITE = -4,  /* NaN or Inf met in a right-hand side or a residual norm */
  LQCD_ERR_SINGULAR = -5,   /* a 6x6 site block of A(x) has no stable inverse */
  LQCD_ERR_STATE = -6       /* call out of order (e.g. apply before set_gauge) */
};

typedef enum {
  LQCD_C64 = 1,    /* complex64: FP32 storage and arithmetic */
  LQCD_C128 = 2,   /* complex128: FP64 storage and arithmetic */
  LQCD_BF16S = 3   /* BF16 storage (re, im pairs), FP32 arithmetic: packed blocks only, see
                      lqcd_pack and lqcd_apply_packed; as solve precision, the Arnoldi basis */
} lqcd_dtype;

typedef enum {
  LQCD_OP_FULL = 0,   /* D on all V sites */
  LQCD_OP_SCHUR = 1   /* S = A_oo - D_oe A_ee^{-1} D_eo on the V/2 odd sites */
} lqcd_op;

typedef enum {
  LQCD_SITES_FULL = 0,
  LQCD_SITES_EVEN = 1,
  LQCD_SITES_ODD = 2
} lqcd_sites;

typedef struct lqcd_ctx_s* lqcd_ctx;

/* Status text ("ok", "invalid argument", ...); static storage, never NULL. */
const char* lqcd_status_string(lqcd_status s);
/* Message of the last failing call on this thread ("" if none); valid until the next call. */
const char* lqcd_last_error(void);

/* Create a lattice context (Sec. III-A-1 lattice and site numbering).
 * dims: host array {T, Z, Y, X}, each even and >= 2, V <= 2^31 / 12 sites.
 * time_bc: +1 or -1. *out receives the handle. No GPU work. */
lqcd_status lqcd_create(const int dims[4], int time_bc, lqcd_ctx* out);
/* Release every device and host resource of ctx; NULL-safe. Synchronises the device. */
lqcd_status lqcd_free(lqcd_ctx ctx);

/* Set the gauge field (Sec. III-A-1, U_mu(x) row-major 3x3 per site and direction).
 * U: host or device, complex128 [V][4][3][3]; read during the call (host: copied
 * synchronously). Builds the library's packed link copies in FP64 and FP32 with
 * the time boundary factor folded into U_0 on the last time slice. Invalidates
 * the site blocks: call lqcd_set_clover() afterwards. */
lqcd_status lqcd_set_gauge(lqcd_ctx ctx, const void* U, void* stream);

/* Set the bare mass m0 and clover coefficient c_sw and build the site blocks
 * A(x) = (4 + m0) - C(x) and A(x)^{-1} (Sec. III-A-1 clover term; the inverse
 * of Sec. III-A-2's odd-even preconditioning) from the current gauge field, in
 * FP64, then their FP32 copies. c_sw = 0 gives the plain Wilson operator (no
 * block arrays are read by the kernels then). Synchronises `stream` to read
 * the singularity flag: LQCD_ERR_SINGULAR if a 6x6 block has a pivot below
 * 1e-14 times its largest entry. */
lqcd_status lqcd_set_clover(lqcd_ctx ctx, double m0, double c_sw, void* stream);

/* Copy the site blocks out for inspection: which = 0 gives A(x), 1 gives A(x)^{-1}.
 * out: device, complex128 [V][12][12] row-major per site, component index
 * 3*spin + colour, sites in canonical order. */
lqcd_status lqcd_export_blocks(lqcd_ctx ctx, int which, void* out, void* stream);

/* Site tile S of the packed layout for nrhs right-hand sides on this lattice: the
 * smallest power of two with S * nrhs >= 16, capped at 16 and at the largest
 * power of two dividing V/2. 0 on bad arguments. */
int lqcd_site_tile(lqcd_ctx ctx, int nrhs);
/* Bytes of one packed spinor block for (dtype, sites, nrhs); 0 on bad arguments. */
size_t lqcd_packed_bytes(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs);

/* Canonical <-> packed conversion of a spinor block (the layout change of
 * Sec. III-A-2's remark that reordering before and after a solve is cheap).
 * in/out: device; canonical complex[nrhs][n_sites][4][3] of `dtype`, packed as
 * described above. For sites = FULL the canonical block lists all V sites in
 * site order; for EVEN/ODD it lists that parity's V/2 sites. For LQCD_BF16S the
 * canonical side is complex64 and the packed side BF16 (rounded to nearest even
 * when packing). */
lqcd_status lqcd_pack(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs,
                      const void* in, void* out, void* stream);
lqcd_status lqcd_unpack(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs,
                        const void* in, void* out, void* stream);

/* eta = op psi on a block of nrhs right-hand sides (Algorithm 1 with the rhs
 * loop inside the site loop, Sec. III-A-1 Eq. (1)-(2)), packed layout.
 * op = FULL: in/out are full-lattice packed blocks (V sites).
 * op = SCHUR: in/out are odd-site packed blocks (V/2 sites); the intermediate
 * A_ee^{-1} D_eo psi lives in library workspace (allocated on first use for
 * this (dtype, nrhs), then reused). in and out must not overlap.
 * dtype LQCD_BF16S: in is a BF16 packed block, out a complex64 packed block,
 * arithmetic (and the Schur intermediate) in FP32; nrhs <= 128.
 * nrhs: 1..256. Requires set_gauge and set_clover. */
lqcd_status lqcd_apply_packed(lqcd_ctx ctx, lqcd_op op, lqcd_dtype dtype, int nrhs,
                              const void* in, void* out, void* stream);

/* Same operator on canonical-layout device blocks: packs, applies, unpacks
 * through library workspace. For LQCD_BF16S, in and out are complex64 blocks and
 * the input is rounded to BF16 when packed. */
lqcd_status lqcd_apply(lqcd_ctx ctx, lqcd_op op, lqcd_dtype dtype, int nrhs,
                       const void* in, void* out, void* stream);

/* Autotuner (not in the paper): times every launch variant of the hopping kernel
 * -- rhs per thread, threads per CTA, minimum resident CTAs (register cap) -- for
 * the full and the Schur operator at this (dtype, nrhs) on library workspace
 * (its contents are arbitrary), and keeps the fastest for every later apply and
 * solve on this context. reps: timed launches per variant (median kept).
 * times_ms: optional host array of 2 * n entries receiving, for variant v,
 * [2v] = full and [2v+1] = Schur median milliseconds (NaN where the variant does
 * not fit nrhs); n_variants: optional, receives n. Synchronises `stream`. */
lqcd_status lqcd_tune(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, int reps, double* times_ms,
                      int* n_variants, void* stream);

/* Tuning cache access: the number of hopping-kernel launch variants for a dtype;
 * the variant used for (dtype, nrhs, op) on this context (the tuned one, else the
 * default; -2 on bad arguments); and an explicit choice (e.g. restored from a
 * saved tuning cache; -1 restores the default). LQCD_ERR_ARG if the variant does
 * not fit nrhs (rhs per thread must divide nrhs). No GPU work. */
int lqcd_kernel_variant_count(lqcd_dtype dtype);
/* Reals per link a launch variant reads (18, or 12 for the two-row copy whose third row the
 * kernel rebuilds; either way the same operator to rounding); -1 on bad arguments. */
int lqcd_kernel_variant_link_reals(lqcd_dtype dtype, int variant);
/* Launch shape of a hopping-kernel variant, written to the caller's host array shape[11]:
 * [0] rhs per thread, [1] threads per CTA, [2] minimum resident CTAs per SM, [3] cp.async
 * stages (0: direct loads), [4] rhs count it is compiled for (0: any), [5] L1 prefetch
 * distance in directions, [6] ring-kernel warps per CTA (0: register kernel), [7] ring slots
 * per warp, [8] reals per link, [9] 1 where a single-parity launch gives each CTA a block of
 * target rows (t, z0 .. z0 + rz - 1, y0, y0 + 1) and walks the directions x, y, z, t (the
 * mapping is taken when whole x rows fill the CTA, rz = targets per CTA / X and rz divides Z;
 * else the plain linear site order), [10] cp.async stages of the pipelined kernel (0: not that
 * kernel), which copies each thread's operands of the next directions into shared memory.
 * LQCD_ERR_ARG on a bad dtype, variant or null pointer. */
lqcd_status lqcd_kernel_variant_shape(lqcd_dtype dtype, int variant, int* shape);
int lqcd_get_kernel_variant(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, lqcd_op op);
lqcd_status lqcd_set_kernel_variant(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs, lqcd_op op, int variant);

/* Link storage of the FP32 operator (Sec. III-A-1 stores U_mu(x) as a row-major 3x3
 * matrix; the BF16 form is the precision extension of the mixed solver, not in the paper):
 *   LQCD_LINKS_FP32 (default): FP32 links (18 reals, or the exact two-row copy with the
 *     third row rebuilt where the autotuner picks such a variant);
 *   LQCD_LINKS_BF16: rows 0 and 1 of every link rounded to BF16 (12 reals, 24 bytes), the
 *     third row rebuilt in FP32 as conj(row0 x row1) and multiplied by the time boundary
 *     factor on the last time slice. This changes the operator by O(2^-9) relative: it
 *     applies to lqcd_apply_packed / lqcd_apply with LQCD_C64 or LQCD_BF16S and to the
 *     FP32 inner operator of lqcd_solve (whose FP64 residual, on the FP64 links, still
 *     decides convergence); FP64 applies are unaffected. The clover blocks stay FP64-built.
 * Takes effect for the next call; no GPU work. LQCD_ERR_ARG for an unknown format. */
enum { LQCD_LINKS_FP32 = 0, LQCD_LINKS_BF16 = 1 };
lqcd_status lqcd_set_link_storage(lqcd_ctx ctx, int format);
/* The context's link storage (LQCD_LINKS_*), -1 for a null context. */
int lqcd_get_link_storage(lqcd_ctx ctx);

/* Odd-even source preparation and solution reconstruction (Sec. III-A-2),
 * packed layout, full-lattice blocks hold even then odd sites:
 *   prepare:     bhat_o = b_o - D_oe A_ee^{-1} b_e          (b full, bhat_o odd)
 *   reconstruct: x = (A_ee^{-1} (b_e - D_eo x_o), x_o)      (b full, x_o odd, x full) */
lqcd_status lqcd_schur_prepare(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs,
                               const void* b, void* bhat_o, void* stream);
lqcd_status lqcd_schur_reconstruct(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs,
                                   const void* b, const void* x_o, void* x, void* stream);

/* One block Gram-Schmidt step of the Arnoldi process (Algorithm 2, "one step of
 * Arnoldi"), per rhs: h_i = <v_i, w> for the nvec basis vectors, w <- w - sum_i h_i v_i,
 * repeated once more when reorth != 0 (CGS2; h accumulates both passes), then
 * h_norm = ||w||. basis: device, nvec packed blocks back to back (each
 * lqcd_packed_bytes(dtype, sites, nrhs) bytes); w: device packed block, updated
 * in place. h: device, complex128 [nvec][nrhs]; hnorm: device, double [nrhs].
 * dtype LQCD_BF16S: BF16 basis, complex64 w, FP32 arithmetic (nrhs <= 32, or even
 * nrhs <= 64).
 * nvec: 1..129. Dot products accumulate per thread in the vector precision and
 * across threads in FP64, in a fixed order (deterministic). */
lqcd_status lqcd_orthogonalise(lqcd_ctx ctx, lqcd_dtype dtype, lqcd_sites sites, int nrhs,
                               int nvec, const void* basis, void* w, void* h, void* hnorm,
                               int reorth, void* stream);

typedef struct {
  int op;             /* LQCD_OP_FULL: GMRES on D; LQCD_OP_SCHUR: on S, x_e reconstructed */
  int precision;      /* LQCD_C128: FP64 Arnoldi; LQCD_C64: FP32 operator and Arnoldi
                         inside FP64 restarts (iterative refinement); LQCD_BF16S: as C64
                         with the Arnoldi basis stored in BF16 (CGS2 always; nrhs <= 32
                         or even nrhs <= 64) */
  int restart_len;    /* m, 1..64 */
  int max_restarts;   /* >= 1 */
  double tol;         /* stop when ||b - D x|| <= tol ||b|| (true residual, per rhs) */
  double inner_tol;   /* C64 / BF16S (nested refinement): an inner solve on the correction
                         equation D e = r_outer runs restarted FP32 cycles, each started
                         from the FP32-computed residual r_outer - D (x - x_outer), until
                         that residual is <= inner_tol * ||r_outer|| or stops decreasing;
                         then the FP64 residual r_outer = b - D x is recomputed. A cycle
                         stops when its Arnoldi estimate reaches that bound (never below
                         tol ||b|| / 2). 0: default 1e-4. C128: unused (every restart
                         recomputes the FP64 residual) */
  int x0_given;       /* 1: x holds the initial guess; 0: start from x = 0 */
  int use_graph;      /* 1: replay each Arnoldi cycle as a captured CUDA graph */
  int reorth;         /* Gram-Schmidt of the Arnoldi step: 0: one classical pass (CGS1);
                         1: CGS2, three passes over the basis per step; 2: CGS2 with the
                         re-orthogonalisation delayed by one step, two passes per step
                         (C64 / BF16S with restart_len <= 32 where the streaming
                         Gram-Schmidt kernel takes the block: nrhs <= 32, or even
                         nrhs <= 64; else as 1).
                         A BF16 basis
                         always re-orthogonalises (0 acts as 1) */
  int profile;        /* 1: time operator and Gram-Schmidt launches with CUDA events
                         (use_graph is then ignored) */
  int dagger;         /* 1: solve the adjoint system D^dagger x = b instead, as
                         gamma5 D^{-1} gamma5 b (D^dagger = gamma5 D gamma5, Sec. III-A-1's
                         operator is gamma5-Hermitian); tol and the reported residuals
                         refer to D^dagger */
  int compact;        /* 1: when at an FP64 restart at least max(1, n/8) of the n rhs still
                         in the block have met tol, repack the others into a block of fewer
                         rhs (library workspace) and continue on it, so retired rhs no longer
                         pass through the operator and Gram-Schmidt kernels; the FP64 residual
                         of the new block is recomputed once. 0: retired rhs stay in the block
                         and only stop contributing basis vectors */
  int block;          /* 1: block GMRES (Sec. II's block Krylov solvers; not the paper's
                         method) as the inner solver: every FP64 residual r is followed by
                         one block GMRES(m) cycle on D e = r in FP32 over one Krylov space
                         shared by all rhs (block CGS2 with Cholesky-QR, Householder least
                         squares), ending when every rhs's residual estimate is below
                         max(tol ||b|| / 2, inner_tol ||r||); converged rhs always leave the
                         block. Needs precision LQCD_C64 and nrhs <= 16; reorth and use_graph
                         are ignored; the stream is synchronised after every step */
} lqcd_solve_params;

typedef struct {
  int status;            /* LQCD_OK or LQCD_NOT_CONVERGED */
  int restarts;          /* Arnoldi cycles (GMRES(m) restarts) that ran */
  int iterations;        /* Arnoldi steps, max over rhs */
  double seconds;        /* host wall time of the call */
  double relres_max;     /* max over rhs of the final ||b - D x|| / ||b|| (full operator) */
  /* profile = 1 only (else 0): summed CUDA-event time, count and algorithmic bytes
   * (bytes the operation must move at least once, see the byte model in the
   * documentation) of the Arnoldi steps that ran */
  double op_ms; int op_launches; double op_bytes;          /* inner-precision operator applies */
  double ortho_ms; int ortho_launches; double ortho_bytes; /* Gram-Schmidt steps (all passes) */
  long long kernel_launches;  /* CUDA kernels this call launched, graph nodes included */
  /* optional per-rhs outputs (host arrays of nrhs entries, may be NULL) */
  int* iters_per_rhs;
  double* relres_per_rhs;
  int outer_steps;       /* FP64 true-residual evaluations r = b - D x (the first included) */
  int ortho;             /* Gram-Schmidt that ran (the reorth meaning: 0, 1 or 2) */
} lqcd_solve_stats;

/* Batched restarted GMRES (Algorithm 2), each rhs independent, optionally on the
 * odd-even Schur system (Sec. III-A-2). b, x: host or device (detected),
 * canonical complex128 [nrhs][V][4][3]; x is overwritten with the solution
 * (and read as the initial guess when x0_given). The true residual is
 * recomputed in FP64 at every restart (C128) or after every inner solve (C64,
 * BF16S: mixed-precision iterative refinement, see inner_tol), each rhs retires
 * once it meets tol, and the final full-operator residual is reported in stats.
 * Synchronises `stream` once per restart. Returns LQCD_NOT_CONVERGED if max_restarts is
 * reached, LQCD_ERR_NONFINITE if b or a residual norm is not finite.
 * stats: host, may be NULL. nrhs: 1..64. */
lqcd_status lqcd_solve(lqcd_ctx ctx, const lqcd_solve_params* params, int nrhs,
                       const void* b, void* x, lqcd_solve_stats* stats, void* stream);

/* Gradient of a loss L = sum_i Re <eta_i, x_i> with x_i = D^{-1} b_i with respect to
 * the gauge links, given x and lambda_i = D^{-dagger} eta_i (an lqcd_solve with dagger = 1
 * on eta): dL = -Re <lambda, (dD) x>, from the hopping terms of D (outer products
 * of the projected spinors pi^-+ x with lambda) and, when c_sw != 0, from the clover
 * term (the derivative of every plaquette leaf of Q_mu,nu). Not in the paper (its
 * solver has no adjoint). grad_U is PyTorch's gradient of a real loss for complex
 * entries: dL = Re sum conj(grad_U) dU over the entries of U treated as independent
 * complex numbers (the su(3) force is TA(U grad_U^dagger)). Uses the context's gauge
 * field and c_sw (set_gauge, set_clover first).
 * x, lambda: device, canonical complex128 [nrhs][V][4][3]; grad_U: device, canonical
 * complex128 [V][4][3][3] (the layout of lqcd_set_gauge's input), overwritten.
 * Library workspace: V * 13.5 KB for the clover leaves. Deterministic (fixed-order
 * sums, no atomics). nrhs: 1..256. */
lqcd_status lqcd_force(lqcd_ctx ctx, int nrhs, const void* x, const void* lambda, void* grad_U,
                       void* stream);

/* Batched GMRES over several lattices of uneven size (one lattice context per
 * entry, distinct contexts): the solve of lqcd_solve for every lattice i with
 * params[i], nrhs[i] rhs, b[i] and x[i] (host or device, canonical complex128),
 * stats[i] (may be NULL). Each restart round synchronises `stream` once for all
 * lattices, retires the lattices whose rhs all meet their tolerance, and runs the
 * restart cycles of all remaining lattices as one captured CUDA graph whose
 * branches (one per lattice, on side streams) execute concurrently; the graph is
 * re-captured only when the set of running lattices changes. Per-rhs retirement
 * inside a cycle works as in lqcd_solve. Profiling (params[i].profile) is not
 * available here. Returns the most severe status over the lattices. Not in the paper
 * (its batch is over the rhs of one lattice); nlat: 1..64. */
lqcd_status lqcd_solve_batch(int nlat, const lqcd_ctx* ctxs, const lqcd_solve_params* params,
                             const int* nrhs, const void* const* b, void* const* x,
                             lqcd_solve_stats* stats, void* stream);

/* Allocation-free Schur apply. The paper has no counterpart: this entry point
 * exists for callers that cannot let the library allocate device memory while
 * they run -- applications whose own pool allocator has already reserved almost
 * all of the GPU's memory (a cudaMalloc from the library would fail), that must
 * know their full device-memory footprint up front, or whose latency-critical
 * loops cannot accept the synchronisation a cudaMalloc/cudaFree may cause.
 * It computes exactly what lqcd_apply_packed(ctx, LQCD_OP_SCHUR, ...) computes
 * (same arguments, packed odd-site blocks in/out, same kernels), but keeps the
 * intermediate A_ee^{-1} D_eo psi_o in a fixed device array of
 * lqcd_noalloc_scratch_bytes() bytes (64 MiB) that every GPU loading the library
 * holds until the process exits, and it calls no cudaMalloc, cudaFree or other
 * allocating routine. Requires V/2 * 12 * nrhs * sizeof(complex) <= that size;
 * larger requests return LQCD_ERR_ARG with a message and do nothing.
 * The first call on each device looks up the array's device address (with that
 * device current) and caches it for the rest of the process; make that first
 * call before any stream capture. The cached address stays valid as long as the
 * device's primary context does: after a cudaDeviceReset in the same process the
 * library (every context and this cache) must not be used again. The device that
 * was current at lqcd_set_gauge must be current here (LQCD_ERR_STATE otherwise).
 * All calls share the one array and it keeps the last call's contents (every
 * call overwrites all it reads): calls that overlap on the GPU, e.g. on two
 * streams at once, race and give wrong results. Requires set_gauge and
 * set_clover (which allocate, at set-up). */
lqcd_status lqcd_apply_schur_noalloc(lqcd_ctx ctx, lqcd_dtype dtype, int nrhs,
                                     const void* in, void* out, void* stream);
/* Measured SIMT FMA rate of the current GPU (not in the paper; a roofline denominator for
 * the FP64 kernels, which are bound by it): *tflops receives the best of three timed launches
 * of independent FMA chains, in TFLOP/s (2 flops per FMA), FP64 if f64 != 0 else FP32.
 * Allocates a small scratch buffer; synchronises `stream`. */
lqcd_status lqcd_fma_peak(int f64, double* tflops, void* stream);

/* Size in bytes of the fixed scratch array used by lqcd_apply_schur_noalloc. */
size_t lqcd_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* LQCD_H */
