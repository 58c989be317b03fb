/*
 * diracst.h - C ABI of the GB300 spacetime finite-element Dirac solver.
 *
 * The library discretises the Dirac equation (i gamma^mu d_mu - m) Psi = 0
 * (Sec. 2.1, Eq. 1) on a structured spacetime mesh of Q1 elements
 * (Sec. 2.2, Eqs. 13-16; 1+1, 2+1 or 3+1), treats the t = 0 layer as known
 * initial data and solves the remaining square system
 *     D_w22 Psi_u = -D_w21 Psi_0                         (Sec. 2.1, Eq. 11)
 * with restarted GMRES (Sec. 2.2; Algorithm 1 steps 5-6).  The operator is
 * never assembled: it is applied matrix-free by CUDA kernels.
 *
 * Conventions shared by every call:
 *   - Rows of D_w22 are premultiplied by gamma^0 ("Hamiltonian form"):
 *       A = i D^t (x) I + i sum_k D^k (x) alpha_k - D^0 (x) (m beta + V),
 *     alpha_k = gamma^0 gamma^k, beta = gamma^0 (Appendix A's element
 *     matrices D^t, D^k, D^0).  The solution equals that of the printed form;
 *     GMRES converges only in this one.
 *   - Gamma matrices: 1+1 gamma^0 = diag(1,-1), gamma^1 = [[0,1],[-1,0]]
 *     (Appendix A); 2+1 adds gamma^2 = -i sigma_x; 3+1 is the Dirac
 *     representation.  Spinor components NC = 2 (1+1, 2+1) or 4 (3+1).
 *   - The potential V is potential energy (i d_t Psi = (H_0 + V) Psi), one
 *     value per spatial element, constant in time (Sec. 4.3, Eq. 21).
 *   - Unknown vector layout: index ((((t-1)*nz + z)*ny + y)*nx + x)*NC + c
 *     for unknown time layers t = 1..N_t, complex interleaved (re, im).
 *     FP64 vectors are double pairs (16 B per entry), FP32 vectors float
 *     pairs (8 B).  Axes a mesh does not have count one node.
 *   - Spatial nodes per axis: PERIODIC n_el (nodes 0..n_el-1), OPEN n_el+1
 *     (natural boundary), DIRICHLET n_el-1 (homogeneous values at both ends
 *     are known and removed like the t = 0 layer).
 *   - Device pointers are CUDA device addresses owned by the caller, on the
 *     device current when the mesh was created; "stream" is a cudaStream_t
 *     (NULL = legacy default stream).  Calls enqueue work on that stream and
 *     return without synchronising unless stated.
 *   - Every call returns a status code (DST_OK = 0 on success) and never
 *     aborts the process.  One mesh must not be used by two host threads at
 *     once.
 */
#ifndef DIRACST_H
#define DIRACST_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DST_API __attribute__((visibility("default")))
#else
#define DST_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  No C++ exception crosses this interface: a failed host
 * allocation or host thread start inside a call returns DST_ERR_OOM, with the
 * reason in dst_last_error_detail(). */
enum {
    DST_OK = 0,
    DST_NOT_CONVERGED = 1,   /* solve hit max_iters; psi holds the best iterate */
    DST_ERR_ARG = -1,        /* invalid argument (null pointer, bad size, bad enum) */
    DST_ERR_OOM = -2,        /* device or host allocation (or host thread start) failed */
    DST_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    DST_ERR_NAN = -5,        /* non-finite value met in the right-hand side or residual */
    DST_ERR_STATE = -6       /* required input not set yet (e.g. initial data) */
};

enum { DST_BC_PERIODIC = 0, DST_BC_OPEN = 1, DST_BC_DIRICHLET = 2 };
enum { DST_FP64 = 0, DST_FP32 = 1 };

typedef struct dst_mesh dst_mesh;   /* opaque, owned by the library */

/*
 * Create a structured spacetime mesh (Algorithm 1 step 1).
 *   d       spatial dimension 1, 2 or 3.
 *   n_el    element counts (x, y, z, t); entries beyond d are ignored except
 *           n_el[3] = N_t >= 1.  Periodic axes need n_el >= 1, Dirichlet >= 2.
 *   lo, hi  domain bounds (x, y, z, t), hi > lo on every used axis.
 *   bc      boundary kind per spatial axis (DST_BC_*), entries beyond d ignored.
 *   out     receives the mesh.  Mass defaults to 1, potential to zero; the
 *           initial data must be set before dst_build_rhs / dst_solve.
 * Errors: DST_ERR_ARG, DST_ERR_CUDA (no device), DST_ERR_OOM.
 */
DST_API int dst_create_mesh(int d, const int64_t n_el[4], const double lo[4], const double hi[4],
                    const int bc[3], dst_mesh **out);

/* Free the mesh and every device buffer it holds.  NULL is accepted. */
DST_API int dst_destroy_mesh(dst_mesh *mesh);

/*
 * Sizes: n_spatial_nodes = nodes of one time layer of unknowns,
 * n_unknowns = N_t * n_spatial_nodes * NC complex entries, ncomp = NC.
 * Any output pointer may be NULL.
 */
DST_API int dst_mesh_sizes(const dst_mesh *mesh, int64_t *n_spatial_nodes, int64_t *n_unknowns,
                   int *ncomp);

/* Particle mass m in the free Dirac equation (Sec. 2.1, Eq. 1).  Any finite value. */
DST_API int dst_set_mass(dst_mesh *mesh, double m);

/*
 * Potential energy per spatial element (Sec. 4.3, Eqs. 21 and 23), copied
 * from HOST memory: nel_x * nel_y * nel_z doubles, x fastest, each the value
 * at the element centroid; NULL resets V to zero.  A potential that depends
 * on x only takes the fast separable path; any other takes a general path.
 * Errors: DST_ERR_ARG (non-finite value), DST_ERR_OOM, DST_ERR_CUDA; after
 * DST_ERR_ARG or DST_ERR_OOM the previous potential stays in force.
 */
DST_API int dst_set_potential(dst_mesh *mesh, const double *V_elem);

/*
 * Initial data Psi_0 on the t = 0 layer (the K known spinors of Sec. 2.1,
 * Eq. 8), copied from HOST memory: n_spatial_nodes * NC complex values
 * (2 doubles each), same layout as one time layer of the unknown vector.
 */
DST_API int dst_set_initial_data(dst_mesh *mesh, const double *psi0);

/*
 * Prescribed spinors on Dirichlet walls (Sec. 2.1, Eq. 2: Psi = Psi_0 on the
 * boundary of the domain).  Like the t = 0 layer they are known, so the split
 * of Eq. 11 moves them to the right-hand side: from this call on,
 * dst_build_rhs and dst_solve add -D_w[unknowns, wall nodes] Psi_wall over
 * every time layer to b.  psi_bd is HOST memory with the spinors of time
 * layers t = 0..N_t on the full node grid of each layer, the walls included:
 * (N_t + 1) layers of gz x gy x gx nodes of NC complex values (2 doubles
 * each), layer slowest, then z, y, x, component, where gk = n_el on a
 * periodic axis, n_el + 1 on an open or Dirichlet axis (axes the mesh does not
 * have count 1).  Only the end nodes of Dirichlet axes are read (layer 0's
 * included; the rest of layer 0 comes from dst_set_initial_data); all other
 * entries are ignored.  The mesh keeps a device copy.  NULL restores
 * homogeneous walls (the default).  Errors: DST_ERR_ARG (mesh without a
 * Dirichlet axis, non-finite wall value; the previous data stays), DST_ERR_OOM,
 * DST_ERR_CUDA.  dst_build_rhs then also needs stream-ordered scratch of two
 * vectors of the open-wall grid (DST_ERR_OOM if it cannot get it).
 */
DST_API int dst_set_boundary_data(dst_mesh *mesh, const double *psi_bd);

/*
 * Right-hand side b = -D_w21 Psi_0 (Sec. 2.1, Eq. 11; Algorithm 1 step 5)
 * into the caller's DEVICE FP64 vector b (n_unknowns complex).  Only the
 * first unknown time layer is non-zero; the call writes every entry.
 * Errors: DST_ERR_STATE (no initial data), DST_ERR_ARG, DST_ERR_CUDA.
 */
DST_API int dst_build_rhs(const dst_mesh *mesh, void *b, void *stream);

/*
 * y = A x with A = D_w22 (Sec. 2.1, Eq. 11; element-by-element sum of
 * Sec. 2.2 evaluated as a sum-factorised stencil), x and y DEVICE vectors of
 * n_unknowns complex values in the given precision (DST_FP64: double pairs,
 * DST_FP32: float pairs, arithmetic in that precision).  x and y must not
 * overlap and must be 16-byte aligned (every cudaMalloc / PyTorch allocation
 * is).  Errors: DST_ERR_ARG, DST_ERR_CUDA.
 */
DST_API int dst_apply_operator(const dst_mesh *mesh, int precision, const void *x, void *y,
                       void *stream);

/*
 * Arnoldi projection h = V^H w (the classical Gram-Schmidt inner products of
 * restarted GMRES, Sec. 2.2): V holds nvec DEVICE FP64 complex vectors of
 * length n stored one after another (vector j starts at V + j*n), w one more;
 * h receives nvec complex values (2*nvec doubles) in DEVICE memory.  The sums
 * are reduced in a fixed order (deterministic).  The call allocates its
 * reduction scratch from the stream-ordered allocator.  1 <= nvec <= 64.
 */
DST_API int dst_arnoldi_project(int64_t n, int nvec, const void *V, const void *w, void *h,
                        void *stream);

/*
 * Arnoldi update: w <- w - V h with the same V layout and a DEVICE h of nvec
 * complex values, and nrm2 (DEVICE, one double) <- ||w||^2 after the update.
 */
DST_API int dst_arnoldi_update(int64_t n, int nvec, const void *V, const void *h, void *w,
                       void *nrm2, void *stream);

/*
 * dst_arnoldi_project without any device allocation.  The paper has no
 * counterpart: this call exists for callers that must not allocate device
 * memory - code that runs under a fixed device-memory budget or inside a host
 * framework that owns every device allocation itself, and code on a
 * latency-critical host path where an allocation could stall, fail late or
 * take a lock the caller already holds.  It computes exactly what
 * dst_arnoldi_project computes (same kernels, same reduction order, so the
 * same bits) and the caller still passes V, w and h.
 *
 * Scratch: the reduction partials live in one statically sized device array
 * of the library (1216 x 64 complex doubles = 1,245,184 bytes), which every
 * GPU that loads the library keeps until the process exits.  Limit:
 * 1 <= nvec <= 64 (any n >= 1); larger nvec returns DST_ERR_ARG and
 * dst_last_error_detail() says why.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current
 * and caches it; make that first call before any stream capture.  No call
 * allocates or frees memory.  All calls share the one array, which keeps the
 * last call's contents; each call writes every partial it reads, so nothing
 * needs clearing, but calls that overlap on the GPU (other streams or host
 * threads) race on it and must be serialised by the caller.
 */
DST_API int dst_arnoldi_project_noalloc(int64_t n, int nvec, const void *V, const void *w, void *h,
                                        void *stream);

typedef struct {
    int restart;            /* Krylov dimension m of GMRES(m); 1..64, default 30 */
    int max_iters;          /* total Arnoldi steps across restarts (and refinements) */
    double rtol;            /* stop when ||b - A x|| <= rtol ||b|| (true residual, FP64) */
    int mixed_precision;    /* 0: FP64 GMRES; 1: FP64 iterative refinement around an
                               inner GMRES whose operator apply runs in FP32 */
    double inner_rtol;      /* inner relative tolerance per refinement step (mixed only) */
    int max_refine;         /* cap on refinement steps (mixed only) */
    int use_initial_guess;  /* 1: psi holds x0 on entry; 0: start from zero */
    int profile;            /* 1: time every kernel with CUDA events (one event between
                               consecutive kernels; ~10% overhead on small meshes) */
    int inner_cycles;       /* GMRES(m) cycles per refinement step (mixed only; 0 = until
                               inner_rtol), default 1.  Cycles after the first restart from
                               the inner residual r - A d computed with the FP32 operator; the
                               refinement's residual b - A psi is always FP64 */
    int ortho;              /* Gram-Schmidt (default 0): 0 = classical, second pass only when the DGKS test
                               asks (norm fell below 1/sqrt 2 of its value before the pass);
                               1 = always two classical passes (CGS2); 2 = one classical pass,
                               never reorthogonalised (PETSc's default for GMRES) */
    int mixed_ortho;        /* mixed only: arithmetic of the inner Gram-Schmidt (default 2).  0 = double-FP32
                               (basis stored as FP32 hi/lo planes, 48-bit significand, error-free
                               FP32 products and sums, FP64 reductions),
                               1 = native FP64 (FP64 basis),
                               2 = FP32-stored basis (8 B per entry, half the traffic of 0) with
                               exact FP32 products and compensated sums: inner products of the
                               stored values err by about 2^-40 of ||v|| ||w||, updates are
                               rounded to FP32 once, each new basis vector is rounded to
                               FP32 once; from 1M unknowns the projection and the update are fed by bulk
                               asynchronous copies */
    int method;             /* Krylov method: 0 = restarted GMRES(restart) (default),
                               1 = BiCGSTAB (van der Vorst 1992; FP64 only, mixed_precision
                               must be 0; iters counts BiCGSTAB steps of two applies each) */
    int batch_cta_max;      /* dst_solve_batch only: meshes of at most this many unknowns are
                               solved one CTA each inside a persistent kernel, larger ones by
                               concurrent single-mesh solves; negative = automatic (default) */
    int precond;            /* right preconditioner (DST_PRECOND_*, default NONE).  With one, the
                               inner GMRES becomes flexible GMRES (Saad 1993): each Arnoldi step
                               applies the operator to z_j = M(v_j), the z_j are kept (FP32), and a
                               cycle's correction is Z y.  Needs mixed_precision = 1,
                               mixed_ortho = 2, method = 0.
                               DST_PRECOND_CN_SWEEP2 applies the sweep twice per step,
                               z = M v + M (v - A M v); DST_PRECOND_CN_LEARNED adds the
                               network attached by dst_set_learned_precond to the sweep.  dst_solve_batch honours it for the meshes
                               it solves one by one and ignores it in the persistent kernel */
} dst_solve_opts;

/* Kernel classes of dst_solve_stats' per-class arrays. */
enum {
    DST_K_APPLY64 = 0,      /* operator apply, FP64 */
    DST_K_APPLY32 = 1,      /* operator apply, FP32 */
    DST_K_CAST = 2,         /* FP64 <-> FP32 vector casts around the FP32 apply */
    DST_K_PROJECT = 3,      /* Arnoldi projection h = V^H w (partials + reduction) */
    DST_K_UPDATE = 4,       /* Arnoldi update w -= V h (+ norm), x += V y */
    DST_K_SCALE = 5,        /* basis normalisation */
    DST_K_MISC = 6,         /* residuals, norms, x += d */
    DST_K_RHS = 7,          /* right-hand side */
    DST_K_PRECOND = 8,      /* preconditioner (Crank-Nicolson sweep: scan, FFTs, march) */
    DST_NUM_KERNEL_CLASSES = 9
};

typedef struct {
    int iters;              /* Arnoldi steps (operator applies inside GMRES cycles) */
    int restarts;           /* GMRES cycles completed */
    int refinements;        /* outer refinement steps (mixed only) */
    int status;             /* same value the call returns */
    double rel_resid_true;  /* ||b - A x|| / ||b|| in FP64 at exit */
    double rel_resid_est;   /* last implicit GMRES residual estimate (relative) */
    double seconds;         /* host wall time of the call (includes synchronisation) */
    double bytes_moved;     /* algorithmic device bytes of the kernels launched */
    double launches;        /* kernel launches of the call */
    int reorths;            /* Arnoldi steps that took a second Gram-Schmidt pass */
    double kernel_ms[9];        /* device time per DST_K_* class (opts.profile only, else 0) */
    double kernel_launches[9];  /* kernel launches per class */
    double kernel_bytes[9];     /* algorithmic bytes per class (reads + writes) */
    double kernel_flops[9];     /* algorithmic floating-point operations per class */
} dst_solve_stats;

/* Fill opts with the defaults (restart 30, max_iters 100000, rtol 1e-8,
 * FP64, inner_rtol 1e-4, max_refine 100000, zero initial guess, no
 * profiling, one inner cycle per refinement, classical Gram-Schmidt with a
 * DGKS-selective second pass, inner Gram-Schmidt on an FP32-stored basis in
 * compensated arithmetic, GMRES, no preconditioner). */
DST_API int dst_default_solve_opts(dst_solve_opts *opts);

/*
 * Solve D_w22 psi = -D_w21 Psi_0 (Algorithm 1 step 6) into the caller's
 * DEVICE FP64 vector psi (n_unknowns complex).  The mesh allocates its GMRES
 * workspace on first use and keeps it until destroyed.  Synchronises the
 * stream before returning.  Returns DST_OK, DST_NOT_CONVERGED (psi holds the
 * last iterate), DST_ERR_NAN, DST_ERR_STATE, DST_ERR_ARG, DST_ERR_OOM or
 * DST_ERR_CUDA; stats (may be NULL) is filled in every case it can be.
 */
DST_API int dst_solve(dst_mesh *mesh, const dst_solve_opts *opts, void *psi, dst_solve_stats *stats,
              void *stream);

/*
 * Tile-shape autotuner of the operator apply (no counterpart in the paper:
 * a GPU launch-configuration choice; every shape computes each output from
 * the same neighbours in the same order, so FP64 applies agree bit for bit and
 * FP32 applies to rounding.  The autotuner picks by timing, so a mixed-precision
 * solve is reproducible bit for bit only with a fixed shape: set one with
 * dst_set_apply_variant before the first solve).  1+1 and
 * 2+1 meshes have 3 shapes (0 = the default: 1+1 tiles of 256 nodes x 32
 * time layers, then 128 x 16 and 64 x 8; 2+1 tiles of 32 x 8 nodes x 8 layers,
 * then 32 x 8 x 4 and 16 x 8 x 8); 3+1 meshes have one.  dst_solve runs the
 * autotuner on a mesh's first solve (in its own workspace).
 *
 * dst_tune_apply: times every shape of both precisions on the mesh (3 applies
 * each after a warm-up, on a stream-ordered scratch of 32 bytes per unknown)
 * and keeps the fastest; synchronises `stream`.  DST_ERR_ARG / OOM / CUDA.
 * dst_set_apply_variant: use shape `variant` (0 .. count-1) for `precision`
 * (DST_FP64 / DST_FP32) from now on; marks the mesh tuned.  DST_ERR_ARG for a
 * bad precision or variant.
 * dst_get_apply_variant: the current shape and the number of shapes.
 */
DST_API int dst_tune_apply(dst_mesh *mesh, void *stream);
DST_API int dst_set_apply_variant(dst_mesh *mesh, int precision, int variant);
DST_API int dst_get_apply_variant(const dst_mesh *mesh, int precision, int *variant, int *count);

/*
 * Batched solve: Algorithm 1 step 6 for `count` independent meshes at once,
 * each psi[i] (DEVICE, complex FP64, meshes[i]'s n_unknowns, 16-byte aligned)
 * receiving the solution of its own mesh.  Every mesh must be 1+1 or 2+1, live
 * on the current device, carry initial data (else DST_ERR_STATE) and have an
 * x-only potential or none (a potential varying along y is DST_ERR_ARG).
 * Every mesh gets the mixed-precision refinement of dst_solve (FP64
 * residual, one GMRES(restart) cycle per refinement with the FP32 operator
 * apply, an FP32-stored basis and compensated Gram-Schmidt, FP64 Givens
 * rotations).  Meshes of at most opts->batch_cta_max unknowns are solved by
 * one CTA each inside a single persistent kernel launch per spatial dimension,
 * without host involvement until all of them finish; larger meshes are solved
 * by single-mesh solves running concurrently from worker threads, each on a
 * stream of its own (the meshes must not be used by other threads meanwhile;
 * if no worker thread can be started, the calling thread solves them).
 * Used from opts: restart (1..32), max_iters and max_refine (per mesh), rtol,
 * inner_rtol, ortho, use_initial_guess, batch_cta_max; method must be 0;
 * mixed_precision, inner_cycles, mixed_ortho and profile are ignored.  The
 * persistent kernel's workspace (two FP64 and restart + 1 FP32 vectors per
 * mesh) is stream-ordered; larger meshes keep their own workspaces as with
 * dst_solve.  Synchronises `stream` before returning.  stats[i] (count entries, required) receives each mesh's steps,
 * refinements, status and true residual; seconds is the wall time of the
 * whole call.  Returns the most severe error status of any mesh (a mesh that
 * did not converge reports DST_NOT_CONVERGED in its stats only), or
 * DST_ERR_ARG / DST_ERR_STATE / DST_ERR_OOM / DST_ERR_CUDA for the call.
 */
DST_API int dst_solve_batch(int count, dst_mesh *const *meshes, const dst_solve_opts *opts, void *const *psi,
                            dst_solve_stats *stats, void *stream);

/*
 * Observables of a solution, per unknown time layer t = 1..N_t, by trapezoidal
 * sums over the spatial nodes (Sec. 4.2, Eq. 20; Sec. 4.3, Eq. 25; the charge
 * monitored in Sec. 4.1): psi is a DEVICE FP64 solution (n_unknowns complex,
 * the layout of dst_solve), out a DEVICE array of N_t x 5 doubles, row t-1 =
 *   [ Q, Q_right, M_x, M_y, M_z ]
 * with Q = sum_nodes w |psi|^2, Q_right the part at x > x0 (a node at x0
 * counts one half), M_k = sum_nodes w x_k |psi|^2 (zero for axes the mesh does
 * not have).  So <x_k>(t) = M_k / Q and the transmitted share T = Q_right / Q.
 * Weights w: product over axes of h (periodic, Dirichlet interior nodes) or
 * h with the two end nodes halved (open axes).  Deterministic (fixed order).
 */
DST_API int dst_observables(const dst_mesh *mesh, const void *psi, double x0, void *out, void *stream);

/*
 * Testing hooks.  The paper has no counterpart: these make the library's
 * failure paths reachable from a test on a healthy GPU, with nothing faulted.
 * Process-wide settings, meant for tests only.
 *   DST_TEST_WAIT_LIMIT  value = tries a bulk-copy wait of the Arnoldi
 *                        projection or update makes before giving up; -1 restores the
 *                        standard 2^22.  With 0 every wait gives up at once,
 *                        before its copy can have landed: the kernel stops
 *                        consuming, waits (standard limit) for the copies it
 *                        has in flight, flags the step, and dst_solve returns
 *                        DST_ERR_CUDA naming the wait in dst_last_error_detail().
 *                        Only mixed solves on an FP32-stored basis of at least
 *                        1,000,000 unknowns use those kernels.
 *   DST_TEST_FAIL_ALLOC  value = how many of the following GMRES workspace
 *                        allocations fail as if the device were out of memory
 *                        (dst_solve returns DST_ERR_OOM, the mesh stays usable);
 *                        0 clears.
 * Errors: DST_ERR_ARG for an unknown hook or a value out of range.
 */
enum { DST_TEST_WAIT_LIMIT = 1, DST_TEST_FAIL_ALLOC = 2 };
DST_API int dst_testing_set(int hook, int64_t value);

/*
 * Testing access to the Gram-Schmidt kernels of the mixed solve on an
 * FP32-stored Krylov basis (Sec. 2.2's GMRES; the arithmetic is the library's):
 * V holds nvec DEVICE FP32 complex vectors (float pairs) of length n (n even,
 * 1 <= nvec <= 64) one after another, w one more.
 *   mode 0: h = V^H w by the register-fed projection (h: DEVICE nvec FP64 complex);
 *   mode 1: the same by the bulk-copy fed projection;
 *   mode 2: w <- w - V h (h: DEVICE FP64 complex input), rounded to FP32 once,
 *           and *nrm2 (DEVICE double) = ||w||^2 of the stored result;
 *   mode 3: the same update with the basis fed by bulk copies;
 *   mode 4: x <- x + V y with x = w read as a DEVICE FP64 complex vector of n
 *           entries and y = h (the end-of-cycle correction; nrm2 unused);
 *   mode 5: the same with the basis fed by bulk copies.
 * Products are exact and sums compensated: the error of h_j is about 2^-40 of
 * ||v_j|| ||w|| (measured with unit basis vectors).  Takes stream-ordered
 * scratch; modes 1, 3 and 5 synchronise the stream.  Errors: DST_ERR_ARG, DST_ERR_OOM,
 * DST_ERR_CUDA (a bulk-copy wait that gave up).
 */
DST_API int dst_testing_fp32_arnoldi(int mode, int64_t n, int nvec, const void *V, void *w, void *h, void *nrm2,
                                     void *stream);

/*
 * Right preconditioners for flexible GMRES (dst_solve_opts.precond).  The paper
 * names none; its conclusion (Sec. 5) asks for one and points at decomposing
 * the time direction.
 *   DST_PRECOND_CN_SWEEP  the Crank-Nicolson sweep M = B^-1 S^-1: S averages
 *     adjacent time layers (S = (I + U) / 2, U the shift to the next layer, the
 *     last layer keeping 1/2) and B is the block lower-bidiagonal
 *     Crank-Nicolson march B[t,t] = i M_s + (h_t/2) K_s, B[t,t-1] = -i M_s +
 *     (h_t/2) K_s, with M_s the spatial mass matrix and K_s the spatial part of
 *     Eq. 7's operator (Appendix A's element matrices).  Meshes whose spatial axes
 *     are all periodic with a constant potential (1+1, 2+1), or whose x axis is
 *     Dirichlet, the others periodic and the potential depends on x only
 *     (1+1, 2+1, 3+1).  Other meshes: DST_ERR_ARG.
 * dst_precond_apply: z = M v for DEVICE FP32 complex vectors v, z of
 * n_unknowns entries (float pairs, the unknown layout), distinct; arithmetic in
 * FP32 (the precision of the inner solve), the layer-solve factors in FP64
 * rounded to FP32.  Takes stream-ordered scratch of about one FP32 vector (plus
 * the factors, 32 NC^2 bytes per x node and frequency, on Dirichlet-x meshes).
 * kind DST_PRECOND_CN_SWEEP, DST_PRECOND_CN_LEARNED (the sweep plus the
 * learned correction below, with the network attached to the mesh by
 * dst_set_learned_precond; two more FP32 vectors of scratch), or
 * DST_PRECOND_BLOCK_JACOBI:
 *   DST_PRECOND_BLOCK_JACOBI  z = blockdiag(A_nn)^-1 v, A_nn the NC x NC block of
 *     D_w22 coupling the components of unknown node n with themselves: the
 *     classical comparator.  Any mesh.  The blocks are read off the operator by
 *     probing (colours of nodes two steps apart along some axis, one FP32 apply
 *     per colour and component, 3^(d+1) x NC applies on meshes whose periodic
 *     lengths are multiples of 3), inverted in FP64 and kept in FP32 by the mesh
 *     (NC^2 complex FP32 per node) until its mass or potential changes; a
 *     singular block is replaced by the identity.  The first use synchronises.
 * Errors: DST_ERR_ARG (kind, mesh not covered, no network attached),
 * DST_ERR_OOM, DST_ERR_CUDA.
 */
enum {
    DST_PRECOND_NONE = 0,
    DST_PRECOND_CN_SWEEP = 1,
    DST_PRECOND_CN_SWEEP2 = 2,
    DST_PRECOND_CN_LEARNED = 3,
    DST_PRECOND_BLOCK_JACOBI = 4
};
DST_API int dst_precond_apply(const dst_mesh *mesh, int kind, const void *v, void *z, void *stream);

/*
 * Energy per unknown time layer, E(t) = int psi^dagger H psi dx with the free
 * Dirac Hamiltonian H = alpha . p + beta m applied spectrally (the energy of
 * Sec. 4.1's conservation study; the paper does not define its E(t), this is
 * one reading of it): FP64 FFT of every layer, then (prod_k h_k) / N times the
 * sum over frequencies of psi^ dagger H(p) psi^, p_k = 2 pi q_k / (n_k h_k) with
 * q_k the signed frequency.  Meshes whose spatial axes are all periodic (axes
 * up to 4096 nodes).  psi: DEVICE FP64 solution (n_unknowns complex); out:
 * DEVICE array of N_t doubles.  Takes stream-ordered scratch of one (3+1: two)
 * FP64 vectors.  Errors: DST_ERR_ARG (a non-periodic axis), DST_ERR_OOM,
 * DST_ERR_CUDA.
 */
DST_API int dst_energy(const dst_mesh *mesh, const void *psi, void *out, void *stream);

/*
 * Learned correction of the sweep (DST_PRECOND_CN_LEARNED; no counterpart in
 * the paper, whose conclusion (Sec. 5) asks for a preconditioner):
 *     M(v) = M_CN(v) + alpha U(rho / s),   rho = v - A M_CN(v),  s = ||rho||,
 * with alpha the complex scale minimising ||rho - alpha A U(rho / s)||, taken
 * afresh for every v (so no corrected direction leaves a larger residual than
 * the sweep alone; one more FP32 operator apply per step), and U a
 * convolutional U-Net on the spacetime node grid (t, [z], [y], x) of the
 * unknowns, 2 NC channels (Re, Im of each spinor component, i.e. the FP32
 * complex unknown vector read as [node][channel] floats).  Layers, in order
 * (conv3: kernel 3 in every grid axis, zero padding keeping the size; conv1:
 * kernel 1; every convolution has a bias):
 *   e1a conv3 C->16 ReLU, e1b conv3 16->16 ReLU (=s1), mean-pool 2;
 *   e2a conv3 16->32 ReLU, e2b conv3 32->32 ReLU (=s2), mean-pool 2;
 *   e3a conv3 32->64 ReLU, e3b conv3 64->64 ReLU, nearest upsample;
 *   u2p conv1 64->32, + s2, u2c conv3 32->32 ReLU, nearest upsample;
 *   u1p conv1 32->16, + s1, u1c conv3 16->16 ReLU; out conv1 16->C.
 * (pooling counts cells past an odd end as zero.)  Convolutions run on BF16
 * tensor cores with FP32 accumulation; parameters are FP32, rounded to BF16.
 * The flat parameter vector holds, per layer in this order, the weight
 * (c_out, c_in, kernel offsets row-major over the grid axes) and then the bias.
 *
 * dst_unet_create: a network for the mesh's grid, parameters zero; DEVICE
 *   memory for parameters, Adam moments, activations and their gradients.
 * dst_unet_num_params / set_params / get_params: the flat FP32 vector (HOST).
 * dst_unet_forward: y = gamma ||x|| U(x / ||x||), x and y DEVICE FP32 complex
 *   vectors of the mesh's n_unknowns entries (distinct).
 * dst_unet_loss_grad: for DEVICE x, target: L = ||U(x^) - t^||^2 / ||t^||^2 with
 *   x^ = x / ||x||, t^ = target / ||x||; *loss (HOST) and the gradient of L with
 *   respect to every parameter (HOST, num_params floats; either may be NULL).
 *   Synchronises the stream.
 * dst_unet_train: `steps` Adam steps (learning rate lr, beta 0.9 / 0.999) on
 *   pairs the method generates on the GPU: e standard normal (splitmix64 of
 *   seed and index), r = A e, z = M_CN(r), input rho = r - A z, target e - z;
 *   loss per step into loss_host (HOST, `steps` floats, may be NULL).  Then the
 *   output scale gamma of dst_unet_forward is set to the least-squares factor
 *   <U, t> / ||U||^2 over 8 fresh pairs (0 if negative): a summary of how well
 *   the network fits the error on such pairs (the solver takes its own scale
 *   per application, above).  The mesh must be one the sweep covers.
 *   Synchronises.
 * dst_unet_output_scale: the current gamma (1 after create / set_params).
 * dst_set_learned_precond: use `net` (NULL: none) in solves of this mesh with
 *   precond = DST_PRECOND_CN_LEARNED.  The mesh does not own it; solves that
 *   share one network must not overlap.
 * Errors: DST_ERR_ARG (a network built for another mesh, bad sizes),
 * DST_ERR_OOM, DST_ERR_CUDA.
 */
typedef struct dst_unet dst_unet;
DST_API int dst_unet_create(const dst_mesh *mesh, dst_unet **out);
DST_API int dst_unet_destroy(dst_unet *net);
DST_API int dst_unet_num_params(const dst_unet *net, int64_t *n);
DST_API int dst_unet_set_params(dst_unet *net, const float *params);
DST_API int dst_unet_get_params(const dst_unet *net, float *params);
DST_API int dst_unet_forward(dst_unet *net, const void *x, void *y, void *stream);
DST_API int dst_unet_loss_grad(dst_unet *net, const void *x, const void *target, double *loss, float *grad,
                               void *stream);
DST_API int dst_unet_train(dst_unet *net, dst_mesh *mesh, int steps, float lr, uint64_t seed, float *loss,
                           void *stream);
DST_API int dst_unet_output_scale(const dst_unet *net, double *gamma);
DST_API int dst_set_learned_precond(dst_mesh *mesh, dst_unet *net);

/* Static, human-readable name of a status code. */
DST_API const char *dst_status_string(int status);

/* Text of the last CUDA failure seen by this host thread (call, file, line,
 * CUDA message) after a DST_ERR_CUDA return; empty if there was none.  The
 * pointer stays valid until the next failing call on the same thread. */
DST_API const char *dst_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* DIRACST_H */
