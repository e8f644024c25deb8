/*
 * nm.h - C ABI of the GB300 filtered-Lanczos normal-mode solver.
 *
 * What it solves. Interior eigenpairs of the continuous-Galerkin P2
 * discretisation of the elastic(-gravitational) equations on a tetrahedral
 * planet mesh (paper Sec. 4, Table of matrix formulae, Appendix A):
 *
 *     K_eff u = lambda M u,  lambda = omega^2 in a slice [lo, hi]      (eq. gep)
 *     K_eff = A_G - E_G A_p^{-1} E_G^T      (Cowling operator, eq. cowling)
 *
 * by a Chebyshev polynomial filter and block Lanczos (Sec. 6.2, which
 * touches A, M and M^{-1} only through matrix-vector products), and, for
 * a rotating body, the projection of the quadratic problem onto the Ritz
 * vectors (eq. sublinear0, Sec. 7).
 *
 * Conventions shared by every call.
 *  - Return value: NM_OK (0) or one of the NM_E* codes below. Nothing
 *    aborts, traps or throws across the ABI; nm_last_error() gives text.
 *  - Objects created by the library (nm_ctx, nm_problem, nm_result) are
 *    owned by it and freed only by the matching *_destroy / *_free call.
 *  - Device pointers passed in are borrowed: the caller allocates them and
 *    keeps them alive for the duration of the call (until the stream
 *    reaches the call's last kernel for the asynchronous calls).
 *  - Blocks of vectors are ROW-MAJOR with a leading dimension: a block of b
 *    vectors over the n = 3 Nu displacement dofs is an (n x b) array with
 *    element (dof i, vector j) at X[i * ld + j], ld >= b. Dof i is
 *    component (i % 3) of u-node (i / 3) in the library's INTERNAL node
 *    order (see nm_problem_unodes); pressure-sized blocks likewise over
 *    the Np pressure nodes.
 *  - Streams: calls that take a cudaStream_t (passed as void*) only
 *    enqueue work on it; NULL means the legacy default stream. Calls
 *    without a stream argument (assembly, lanczos_slice, ritz) run on the
 *    problem's own stream and return after synchronising it.
 *  - Precision: NM_F64 computes in double, NM_F32 in float (values and
 *    accumulators), for the filter-path calls that take an nm_prec.
 */
#ifndef NM_H
#define NM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    NM_OK = 0,
    NM_EINVAL = 1,        /* invalid argument or malformed mesh             */
    NM_ENOMEM = 2,        /* device or host allocation failed               */
    NM_ENOTCONV = 3,      /* solver stopped without converging              */
    NM_ECUDA = 4,         /* a CUDA / cuBLAS / cuSOLVER call failed          */
    NM_ETIMEOUT = 5,      /* a bounded device wait ran out                  */
    NM_EUNSUPPORTED = 6   /* option not supported by the library            */
};

/* NM_F64: every step in double. NM_F32: the whole filter recurrence in
 * float. NM_MIXED: double recurrence and K_eff SpMMs; each inner solve (mass
 * and fluid pressure) is k steps of float semi-iteration, one double
 * residual r = w - A x (float iterate, double values and sums), and k more
 * float steps on r, so the applied inverse is accurate to ~(2 rho^k)^2
 * while its vectors carry double rounding only. Blocks are double. */
typedef enum { NM_F64 = 0, NM_F32 = 1, NM_MIXED = 2 } nm_prec;
typedef enum { NM_UNIT_OMEGA = 0, NM_UNIT_OMEGA2 = 1 } nm_unit;
typedef enum { NM_RITZ_PENCIL = 0, NM_RITZ_ROTATING = 1 } nm_ritz_mode;

/* flags of nm_model */
#define NM_GRAVITY       1u   /* include the reference-gravity terms of A_G and E_G */
#define NM_CENTRIFUGAL   2u   /* g' = g - grad psi: not supported (NM_EUNSUPPORTED) */
/* Self-gravitation: the full operator K_eff - C^T S C of Sec. 5.2 (eqs.
 * ph1body2, ph1surface2, phi1fluidsolid, eigfull) instead of the Cowling
 * approximation. C maps u to the point masses of the elements
 * (rho_k int_K div u at the barycentre) and of the outer-boundary and
 * fluid-solid faces (the density jump times int_E nu . u, at the face
 * barycentre); S is G / |r_i - r_j| between points and G / R_i on the
 * diagonal, 1/R_i the mean of 1/|x - r_i| over the point's own element or
 * face. Applied by a direct FP64 sum over the points (O(points^2) per
 * column, points ~ tets + boundary faces; its point buffers, 2 * 64
 * doubles per point, are allocated at assembly). Supported with NM_F64 and
 * NM_MIXED (the term is applied in double); NM_F32 products return
 * NM_EUNSUPPORTED. */
#define NM_SELF_GRAVITY  4u

typedef struct nm_ctx nm_ctx;
typedef struct nm_problem nm_problem;
typedef struct nm_result nm_result;
typedef struct nm_lanczos nm_lanczos;

/* Mesh (host memory, read during nm_assemble only).
 * xyz[3*nv] vertex coordinates; tet[4*nt] vertex ids (0-based, any
 * orientation, non-degenerate); region[nt]: 0 solid, 1 fluid. */
typedef struct {
    int64_t nv;
    const double* xyz;
    int64_t nt;
    const int32_t* tet;
    const uint8_t* region;
} nm_mesh;

/* Model (host memory, read during nm_assemble only). Per-tet constants
 * (Appendix A samples rho, c, kappa, N^2 per element): rho > 0, Lame
 * lambda and mu (fluid: mu = 0, kappa = lambda), N2 (fluid buoyancy).
 * gprime: optional reference field g' at the CANONICAL P2 nodes (3 * n_p2
 * doubles, canonical order as in nm_problem_unodes); NULL = computed by
 * direct summation over tet point masses with constant G (Sec. 5.1).
 * Omega: rotation vector used by NM_RITZ_ROTATING (c_r, eq. rotationQ). */
typedef struct {
    const double* rho;
    const double* lam;
    const double* mu;
    const double* N2;
    const double* gprime;
    double G;
    double Omega[3];
    uint32_t flags;
} nm_model;

typedef struct {
    int64_t nv, nt;
    int64_t n_p2;      /* P2 nodes: vertices + edges                       */
    int64_t Nu;        /* displacement nodes (fluid-solid nodes twice)      */
    int64_t n;         /* displacement dofs = 3 Nu                          */
    int64_t Np;        /* pressure nodes (0 without fluid)                  */
    int64_t nnz_u;     /* stored blocks of A_G (= stored entries of M_rho)  */
    int64_t nnz_p;     /* stored entries of A_p                             */
    int64_t nnz_e;     /* stored 3x1 blocks of E_G                          */
    int64_t n_fs;      /* fluid-solid interface faces                       */
    int64_t n_charges; /* charge points of NM_SELF_GRAVITY (0 without it)   */
} nm_problem_info;

/* Filter for nm_filter_apply: Z = sum_{k=0..degree} gamma[k] T_k(B) Y with
 * B = (P_M K_eff - c)/e, T_k Chebyshev polynomials, P_M ~ M^{-1} by k_M
 * steps of Jacobi-preconditioned Chebyshev semi-iteration with bounds
 * [m_lo, m_hi] of D^{-1} M, and the A_p^{-1} of K_eff by k_P steps with the
 * same bounds. gamma: host array of degree+1 doubles. */
typedef struct {
    int32_t degree;
    const double* gamma;
    double c, e;
    int32_t k_M, k_P;
    double m_lo, m_hi;   /* 0, 0: the P2 element bounds [1/4, (19+sqrt 249)/8] */
} nm_filter;

typedef struct {
    int32_t block;        /* Lanczos block width b (1..64)                   */
    int32_t degree;       /* filter degree d                                 */
    int32_t k_M, k_P;     /* inner semi-iteration steps (0: 57 / 57)         */
    int32_t max_blocks;   /* basis size limit in blocks                      */
    int32_t check_every;  /* Rayleigh-Ritz convergence test period (blocks)  */
    nm_prec filter_prec;  /* precision of the filter SpMMs and mass solves   */
    double tol;           /* residual tolerance (default 1e-6)               */
    uint64_t seed;        /* start block seed (counter-based Philox-4x32-10) */
    const double* start;  /* optional device start block (n x block, ld=block); NULL: drawn from seed */
    int32_t bounds_steps; /* Lanczos steps for the spectrum bounds (0: 40)   */
    int32_t log_every;    /* > 0: one progress line on stderr every that many blocks */
} nm_slice_opts;

/* ---- context ---------------------------------------------------------- */
/* Create a context on CUDA device `device` (cudaSetDevice is called). */
int nm_ctx_create(int device, nm_ctx** out);
int nm_ctx_destroy(nm_ctx* ctx);
/* Last error message of the context (or of the most recent failing call
 * when ctx is NULL). Valid until the next call on that context. */
const char* nm_last_error(const nm_ctx* ctx);

/* ---- assembly (Sec. 4.2, Appendix A) ----------------------------------
 * Builds every matrix on the device and keeps it resident: A_G as a 3x3
 * block CSR over the u-nodes, M_rho as a scalar CSR on the same graph,
 * -A_p as a scalar CSR over the pressure nodes, E_G as 3x1 and E_G^T as
 * 1x3 block CSR. NM_EINVAL on malformed input (ids out of range,
 * degenerate tet, rho <= 0, fluid kappa <= 0). */
int nm_assemble(nm_ctx* ctx, const nm_mesh* mesh, const nm_model* model, nm_problem** out);
int nm_problem_free(nm_problem* prob);
int nm_problem_get_info(const nm_problem* prob, nm_problem_info* info);

/* Node maps (host outputs, caller-allocated):
 * canon[Nu]: the canonical u-node id of each internal u-node. Canonical
 *   order: P2 nodes are the mesh vertices 0..nv-1 then every edge once in
 *   lexicographic (min vertex, max vertex) order; u-nodes are the P2 nodes
 *   touching a solid tet in increasing P2 id, then those touching a fluid
 *   tet in increasing P2 id.
 * p2[Nu]: the P2 node id of each internal u-node (may be NULL).
 * pcanon[Np]: the canonical pressure node of each internal pressure node
 *   (fluid P2 nodes in increasing P2 id; may be NULL). */
int nm_problem_unodes(const nm_problem* prob, int64_t* canon, int64_t* p2, int64_t* pcanon);

/* Copy an assembled matrix to host CSR in the library's internal order.
 * which: 0 A_G (3x3 blocks, vals 9 per block, row-major), 1 M_rho (1 per
 * entry), 2 -A_p, 3 E_G (3x1 blocks), 4 E_G^T (1x3 blocks). Pass NULL
 * buffers to query sizes in *nrows / *nnz; then rowptr[nrows+1],
 * col[nnz], vals[nnz * block entries]. */
int nm_problem_export(const nm_problem* prob, int which, int64_t* nrows, int64_t* nnz,
                      int64_t* rowptr, int32_t* col, double* vals);

/* Tuning knobs of a problem (the autotuner's hooks). key "sched": 1 gives
 * the semi-iteration SpMMs of blocks 17..64 wide an SM-local row order
 * (each SM walks its own contiguous range of Morton-ordered rows, so
 * neighbour gathers hit in L1): the vectorised kernel below takes its row
 * blocks in that order, the others run as persistent SM-local kernels;
 * 0 (default) uses one warp per row over a plain grid. key "chunk": 256,
 * 512 or 1024 runs those SpMMs one warp per row with each CTA sweeping its
 * own contiguous range of rows in a single wave (CTA size = the value, L1
 * preferred over shared memory); 0 (default) turns it off; it takes
 * precedence over the other schedules. key "vec": 1 (default) runs the float semi-iteration SpMMs
 * of blocks exactly 32 wide with ld = 32 with 16-byte vectorised gathers
 * (each row split over four groups of eight lanes), 0 with one 4-byte
 * gather per lane and component; key "vec_threads" (32 default, 64, 128,
 * 256, 512, 1024; one row per warp) sets their CTA size for the
 * 3-component mass rows, "vec_threads_p" (128 default) for the
 * 1-component pressure rows: larger CTAs put more consecutive rows on one
 * SM's L1, smaller ones free their slot sooner when a CTA's rows differ in
 * length. key "df_threads" (32 default, 64, 128, 256): CTA size of the
 * NM_MIXED form's lane-group double-float SpMMs (b = 32). key "overlap":
 * 1 runs the mixed-form K_eff's fluid pressure chain (E_G^T X, the refined
 * A_p solve) on a high-priority second stream of the problem while the A_G
 * product runs on the caller's stream, then adds E_G S; 0 (default) runs
 * them in sequence with E_G S fused into the A_G product. key "graphs": 1
 * replays degrees 1..d-1 of the NM_MIXED filter recurrence from two
 * captured CUDA graphs (odd / even degree; gamma_{k+1} read on the device
 * at a device-side degree counter), on streams other than the legacy
 * default stream and when profiling is off; results are identical to the
 * eager launches. 0 (default) launches every kernel from the host. key "tile_rows": height of the row
 * tiles whose gathered operand the float kernels stage in shared memory
 * (0, the default, disables staging; 4..64, power of two); the tiles are
 * rebuilt on the host. key "tile_kernel": 1 or 2, the staged kernel
 * variant (256-thread rounds / 512-thread unrolled rounds). key
 * "double_float": 1 (default) runs the NM_MIXED form's double-precision
 * SpMMs (the K_eff block SpMM and the refinement residuals) as
 * double-float arithmetic on the float units (values split exactly into
 * two floats, error-free products and sums, ~2^-48 relative); 0 runs them
 * in double. key "tma": 1 runs the float mass steps of 32-column blocks
 * (ld 32) as the shared-memory staged kernel: persistent CTAs whose
 * producer warps copy each row tile's distinct neighbour records into a
 * three-stage shared-memory ring (cp.async, with cp.async.bulk for the
 * tile's index and value windows, completion on mbarriers) while consumer
 * warps compute the previous tiles; the tiles (at most 32 rows and 160
 * distinct neighbours) are built on the host on first use. Its waits are
 * bounded: a wait that runs out makes the next nm_lanczos_step return
 * NM_ETIMEOUT. 0 (default) uses the lane-group kernel. NM_EINVAL for an
 * unknown key or value. */
int nm_set_option(nm_problem* prob, const char* key, int64_t value);

/* Autotuner: times one degree of the filter recurrence (precision prec,
 * block width b, inner steps k_M) on this problem for every kernel variant
 * of the options above ("sched", "chunk", "vec", "tile_rows"/"tile_kernel", and for
 * NM_MIXED "graphs", "tma" and "double_float"), keeps the fastest, and reports the time per
 * column and degree of block widths 16, 32 and 64 with it. All variants
 * compute the same sums (up to rounding order). report: caller buffer
 * (may be NULL) for a one-line JSON summary, truncated to report_len. */
int nm_autotune(nm_problem* prob, int b, nm_prec prec, int k_M, char* report, int report_len);

/* Reference field g' at the internal u-nodes (host out, 3*Nu doubles). */
int nm_problem_gravity(const nm_problem* prob, double* g);

/* ---- operator pieces (A, M, M^{-1} as matrix-vector products, Sec. 6.2) */
/* Y = K_eff X. The fluid Schur term uses k_P steps (0: 80, effectively
 * exact in FP64) of the Jacobi-Chebyshev solve for -A_p. X, Y device. */
int nm_apply_K(nm_problem* prob, const void* X, int64_t ldx, void* Y, int64_t ldy, int b,
               int k_P, nm_prec prec, void* stream);
/* Y = M X (M = M_rho (x) I_3). */
int nm_apply_M(nm_problem* prob, const void* X, int64_t ldx, void* Y, int64_t ldy, int b,
               nm_prec prec, void* stream);
/* X = P_M W: k_M steps of Jacobi-preconditioned Chebyshev semi-iteration
 * for M X = W with bounds [m_lo, m_hi] (0, 0: the P2 element bounds). */
int nm_solve_M(nm_problem* prob, int k_M, double m_lo, double m_hi, const void* W, int64_t ldw,
               void* X, int64_t ldx, int b, nm_prec prec, void* stream);
/* Y = R X with R = M_rho (x) [Omega]_x (Coriolis form c_r, eq. rotationQ;
 * the paper's R_s, R_f with the Levi-Civita symbol contracted with Omega). */
int nm_apply_R(nm_problem* prob, const void* X, int64_t ldx, void* Y, int64_t ldy, int b,
               nm_prec prec, void* stream);

/* ---- slice set-up ------------------------------------------------------
 * Store the target interval (eq. freq): unit NM_UNIT_OMEGA takes angular
 * frequencies (lambda = omega^2; lo <= 0 means lambda_lo = 0), unit
 * NM_UNIT_OMEGA2 takes lambda directly, negative lo included (the full
 * operator of NM_SELF_GRAVITY has negative eigenvalues). lambda_lo = 0 is
 * moved to -1e-8 * lambda_max at solve time so that zero modes are inside.
 * A slice whose negative lambda_lo lies below the estimated bottom of the
 * spectrum widens the Chebyshev map of its run down to that edge. */
int nm_set_interval(nm_problem* prob, double lo, double hi, nm_unit unit);
/* Spectrum bounds of B = P_M K_eff (Lanczos with `steps` steps, FP64):
 * lam_hi = 1.01 (theta_max + |resid|), lam_lo = min(0, theta_min) - 1e-6 lam_hi
 * (the bottom Ritz residual is not subtracted: it is large at the clustered
 * low end and would cost filter resolution where low slices sit). */
int nm_spectrum_bounds(nm_problem* prob, int steps, int k_M, uint64_t seed, double* lam_lo,
                       double* lam_hi);
/* Jackson-damped Chebyshev coefficients of the indicator of [xi, eta]
 * mapped from [lam_lo, lam_hi] to [-1, 1] (host math). gamma[degree+1],
 * c, e out. */
int nm_filter_design(double lam_lo, double lam_hi, double xi, double eta, int degree,
                     double* gamma, double* c, double* e);

/* ---- hot path ------------------------------------------------------------
 * Z = p(B) Y for a block of b vectors (row-major, device). Scratch for the
 * recurrence is owned by the problem and reused across calls (allocated
 * on first use for the largest b seen). prec selects the arithmetic of the
 * whole recurrence; X and Y then hold doubles (NM_F64) or floats (NM_F32). */
int nm_filter_apply(nm_problem* prob, const nm_filter* f, const void* Y, int64_t ldy, void* Z,
                    int64_t ldz, int b, nm_prec prec, void* stream);

/* ---- filter application without device allocation -------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc: a host whose device memory is handed out by
 * another allocator (a framework's pool that has already reserved the free
 * HBM), a serving loop that cannot afford the device synchronisation of
 * cudaMalloc / cudaFree, or a host that must know its full device footprint
 * when the library loads.
 *
 * Computes exactly what nm_filter_apply does with prec = NM_F64 (same
 * kernels in the same order): Z = p(B) Y, Y and Z device arrays of doubles,
 * row-major n x b with leading dimensions ldy, ldz >= b, owned by the
 * caller. The recurrence scratch, (5 n + 3 Np) * b * 8 bytes, lives in a
 * file-scope device array of NM_STATIC_SCRATCH_BYTES; the call allocates
 * no device memory (no cudaMalloc, cudaFree or allocating library call).
 *  - Sizes whose scratch exceeds NM_STATIC_SCRATCH_BYTES are rejected with
 *    NM_EINVAL and a message giving the bytes needed; nothing is launched.
 *  - Every GPU on which the call runs holds the array until process exit.
 *  - All calls on one device share the array, which keeps the last call's
 *    contents (each call clears the bytes it uses on its stream before
 *    the recurrence). Calls whose kernels overlap on the GPU (different
 *    streams, threads, contexts or problems) race on it: serialise them.
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress and keeps it for the life of the process; make
 *    that first call before any stream capture. The kept address does not
 *    survive cudaDeviceReset (or any other end of the device's primary
 *    context) in the same process: do not call this entry point on a
 *    device after resetting it.
 *  - Not recorded by nm_profile. Other errors as nm_filter_apply. */
#define NM_STATIC_SCRATCH_BYTES (16u << 20)
int nm_filter_apply_static(nm_problem* prob, const nm_filter* f, const double* Y, int64_t ldy, double* Z,
                           int64_t ldz, int b, void* stream);

/* Filtered block Lanczos for every eigenpair with lambda in the interval
 * set by nm_set_interval (Sec. 6.2), followed by an FP64 Rayleigh-Ritz of
 * the pencil and FP64 residuals. The slice has converged when every Ritz
 * value of the filtered operator above the threshold has converged and
 * the slice's pencil pairs in their span pass tol; it is converged and
 * empty (k = 0) when, at two consecutive checks from the fourth block on,
 * those Ritz values have converged and no pair lies in the slice.
 * NM_ENOTCONV if max_blocks is reached first (the result is still
 * returned). */
int nm_lanczos_slice(nm_problem* prob, const nm_slice_opts* opts, nm_result** out);

/* Batched slices: nslices slices (lo[i], hi[i] in the given unit, as in
 * nm_set_interval) solved in lockstep with one filter recurrence per block
 * step over the concatenated blocks (up to 64 columns per recurrence: more
 * slices are filtered in groups of 64 / block slices; the
 * slices share the spectrum bounds and the Chebyshev map, each keeps its
 * own coefficients, basis, reorthogonalisation, convergence test and
 * Rayleigh-Ritz). out: caller array of nslices result pointers.
 * NM_ENOTCONV if any slice stops at max_blocks (every result is returned). */
int nm_lanczos_multi(nm_problem* prob, const nm_slice_opts* opts, int nslices, const double* lo, const double* hi,
                     nm_unit unit, nm_result** out);

/* ---- resumable block Lanczos ----------------------------------------------
 * The filtered block Lanczos of nm_lanczos_slice / nm_lanczos_multi
 * (Sec. 6.2) split into its block steps, so that a caller can interleave
 * slices, bound the work per call, or stop early:
 *
 *   nm_lanczos_begin  spectrum bounds of P_M K_eff (reused when the problem
 *                     already holds bounds for the same bounds_steps, k_M
 *                     and seed + 1; any nm_set_option clears them), the
 *                     filter of each slice, the start block (opts->start,
 *                     read during this call only, else Philox from seed)
 *                     and its Cholesky-QR in the M inner product.
 *                     nslices = 0 takes the one interval of nm_set_interval
 *                     (lo, hi, unit ignored); else as nm_lanczos_multi.
 *   nm_lanczos_step   one block step of every active slice: filter the
 *                     current blocks (one recurrence over the concatenated
 *                     blocks), two-pass CGS and Cholesky-QR of each new
 *                     block, the projected block-tridiagonal matrix; every
 *                     check_every blocks (and at max_blocks) the Ritz
 *                     convergence test and, when every wanted Ritz value of
 *                     p(B) has converged, the FP64 Rayleigh-Ritz of the
 *                     pencil; a slice whose Ritz pairs all pass tol stops.
 *                     *active = slices still running (0: call finish).
 *   nm_lanczos_get_info progress of slice i (host copy, no synchronisation).
 *   nm_lanczos_add    a slice joins the running batch (continuous batching):
 *                     its filter on the run's spectrum bounds, degree and
 *                     options, its start block (start: device n x block,
 *                     ld block, read during this call; NULL: Philox from
 *                     seed) and its Cholesky-QR; it takes block steps from
 *                     the next nm_lanczos_step on, with its own block
 *                     counter. *index = its slice number (slices are
 *                     numbered in the order they were begun or added).
 *   nm_lanczos_take   the result of one slice, which leaves the run (its
 *                     basis is released); a slice still running is stopped
 *                     with a Rayleigh-Ritz on its current basis and
 *                     NM_ENOTCONV (the result is returned all the same).
 *   nm_lanczos_finish the results of every slice not taken yet (out:
 *                     caller array with one pointer per slice begun or
 *                     added; taken slices get NULL; a Rayleigh-Ritz on the
 *                     current basis of a slice that has none yet).
 *                     NM_ENOTCONV if a slice did not pass tol; the results
 *                     are returned all the same and belong to the caller
 *                     (nm_result_free).
 *   nm_lanczos_free   releases the run (its bases); call after finish, or
 *                     instead of it to abandon the run.
 *
 * Running begin, step until *active == 0, finish computes exactly what
 * nm_lanczos_multi computes. The run borrows the problem: free it before
 * the problem, and use one run of a problem at a time from one thread. */
typedef struct {
    int32_t blocks;          /* block steps taken by this slice             */
    int32_t m;               /* basis columns                               */
    int32_t active;          /* 1 while the slice takes further steps       */
    int32_t converged;       /* 1 once its Rayleigh-Ritz pairs pass tol      */
    int32_t wanted;          /* Ritz values of p(B) above the threshold      */
    int32_t ritz_converged;  /* ... whose residual estimate passed           */
    double seconds_filter;   /* filter time of the run so far               */
} nm_lanczos_info;

int nm_lanczos_begin(nm_problem* prob, const nm_slice_opts* opts, int nslices, const double* lo, const double* hi,
                     nm_unit unit, nm_lanczos** out);
int nm_lanczos_step(nm_lanczos* run, int* active);
int nm_lanczos_get_info(const nm_lanczos* run, int slice, nm_lanczos_info* info);
int nm_lanczos_add(nm_lanczos* run, double lo, double hi, nm_unit unit, uint64_t seed, const double* start,
                   int* index);
int nm_lanczos_take(nm_lanczos* run, int slice, nm_result** out);
int nm_lanczos_finish(nm_lanczos* run, nm_result** out);
int nm_lanczos_free(nm_lanczos* run);

/* Rayleigh-Ritz on a caller basis V (device, n x m, row-major, ld ldv,
 * FP64). NM_RITZ_PENCIL: Ritz pairs of (K_eff, M) on span V inside the
 * interval. NM_RITZ_ROTATING: V must hold M-orthonormal Ritz vectors X_e
 * with Ritz values lam_e (host, m doubles, all > 0); solves the projected
 * rotating problem (eq. sublinear0) and keeps omega in [w_lo, w_hi] of
 * the interval (unit omega). */
int nm_ritz(nm_problem* prob, nm_ritz_mode mode, const double* V, int64_t ldv, int m,
            const double* lam_e, nm_result** out);

/* ---- dense products -------------------------------------------------------
 * The dense algebra of the block Lanczos and the Ritz projections (Sec. 6.2:
 * the Gram-Schmidt coefficients V^T M W and updates W - V C; Rayleigh-Ritz
 * V^T K V, V^T M V and X = V S; Sec. 7: X^T R X) in FP64 accuracy on the
 * tensor cores: each operand is cut into eight exact 7-bit pieces per
 * chunk of 64 contraction terms (scaled to the largest entry of its row or
 * column in the chunk), the 36 leading piece products run as bf16 tensor-
 * core products with exact float accumulation, and the chunk sums are
 * added in FP64. The error is of the order of 2^-53 times the sum over the
 * contraction of the products of each row's and column's largest entries.
 * Deterministic (fixed split and summation order). All pointers device.
 * nm_gemm_tn: C (I x J, column-major, ld ldc) = alpha X^T Y + beta C with
 *   X (K x I) and Y (K x J) row-major (ld ldx, ldy); the split parts of the
 *   contraction use a workspace the context owns (grown on demand).
 * nm_gemm_nn: D (I x J, row-major, ld ldd) = alpha X Y + beta D with X
 *   (I x K) row-major (ld ldx) and Y (K x J) column-major (ld ldy).
 * beta = 0 does not read C / D. NM_EINVAL for negative sizes or leading
 * dimensions too small. Problems use these products unless the option
 * "dense_tc" of nm_set_option is 0 (cuBLAS DGEMM then). */
int nm_gemm_tn(nm_ctx* ctx, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
               const double* Y, int64_t ldy, double beta, double* C, int64_t ldc, void* stream);
int nm_gemm_nn(nm_ctx* ctx, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
               const double* Y, int64_t ldy, double beta, double* D, int64_t ldd, void* stream);

/* ---- kernel timing --------------------------------------------------------
 * With profiling enabled, every filter degree brackets its launch
 * sequences with CUDA events on the launching stream: kind 0 = the mass
 * solve (NM_F64 / NM_F32: its k_M - 1 back-to-back launches of the fused
 * M_rho SpMM + update kernel; NM_MIXED: the whole refined solve, 2 k_M + 3
 * launches), kind 1 = the K_eff application (E_G^T SpMM, the pressure
 * semi-iteration, the A_G (+ E_G) SpMM), kind 2 = NM_MIXED only: the
 * float M_rho semi-iteration launches alone (k_M - 1 back-to-back launches
 * per half of each refined mass solve).
 * nm_profile_read synchronises the problem's recorded streams and returns
 * the launch count and summed device milliseconds of a kind since the
 * last reset. Profiling adds two events per region and degree. */
int nm_profile(nm_problem* prob, int enable, int reset);
/* Number of kernels this library has launched in the process so far
 * (every launch of every entry point, all devices). */
uint64_t nm_kernel_launches(void);
int nm_profile_read(nm_problem* prob, int kind, int64_t* launches, double* ms);

/* ---- results ------------------------------------------------------------ */
typedef struct {
    int64_t k;            /* eigenpairs returned                              */
    int64_t n;            /* rows of the eigenvector block                    */
    int32_t complex_vectors; /* 1: X holds complex128 (rotating), else float64 */
    int32_t blocks;       /* Lanczos blocks used                               */
    int64_t m;            /* basis columns used                                */
    int64_t filter_applications; /* vectors filtered (blocks x b)             */
    double lam_lo, lam_hi;/* spectrum bounds used                               */
    double seconds;       /* wall time of the call                             */
    double seconds_filter;/* part spent in nm_filter_apply                     */
} nm_result_info;

int nm_result_get_info(const nm_result* res, nm_result_info* info);
/* Host copies: lambda[k] (lambda = omega^2; rotating: omega), resid[k]. */
int nm_result_values(const nm_result* res, double* lambda, double* resid);
/* Device pointer of the eigenvector block (n x k row-major, ld = k), owned
 * by the result. */
const void* nm_result_vectors(const nm_result* res);
int nm_result_free(nm_result* res);

#ifdef __cplusplus
}
#endif

#endif /* NM_H */
