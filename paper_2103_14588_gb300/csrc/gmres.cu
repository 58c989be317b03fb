// Restarted GMRES(m) and FP32-apply iterative refinement around it
// (Algorithm 1 step 6: "solve the linear system by utilizing KSP"; the
// Krylov method is GMRES, Saad & Schultz 1986, named in Sec. 2.2).
//
// Arnoldi uses classical Gram-Schmidt: one pass is a projection h = V^H w and
// an update w <- w - V h over the whole basis (two streams over V instead of
// one per basis vector as in modified Gram-Schmidt).  A second pass is made
// when the DGKS test asks for it (Daniel, Gragg, Kaufman & Stewart 1976: the
// norm after the pass fell below 1/sqrt(2) of the norm before), or always
// (CGS2) on request.  The Hessenberg column goes to the host, which applies
// the Givens rotations and tracks the least-squares residual |g_{j+1}|.  Every
// restart recomputes the true residual b - A x in FP64.
//
// Mixed precision (iterative refinement): the outer loop keeps x, the
// residual r = b - A x and the convergence test in FP64; each correction d
// solves A d = r approximately with the same GMRES, whose operator apply
// runs in FP32 (inputs rounded to FP32, output widened back to FP64), while
// orthogonalisation, Givens rotations and the least-squares update stay FP64.
// By default a correction is a single GMRES(m) cycle (or less, if it reaches
// the inner tolerance), so the refinement is restarted GMRES whose restart
// residual is recomputed with the FP64 operator; with inner_cycles > 1 the
// later cycles of a correction restart from the inner residual computed with
// the FP32 operator.
//
// The host marks the phases of a solve with NVTX ranges ("dst_solve", its
// setup, each GMRES cycle, the FP64 refinement residual, the FP32 inner
// residual) for timeline tools; without one attached they cost nothing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "blas.h"
#include "internal.h"
#include "sweep.h"

namespace {

using cplx = std::complex<double>;

// a named host range for timeline tools (NVTX)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Workspace {
    int64_t n;
    int m;
    bool mixed;
    double2 *V, *b, *tmp, *d, *r64, *rin, *h1, *h2;   // rin: inner residual between cycles of one refinement
    float2 *x32, *y32;
    double *nrm;
    unsigned *tickets;     // [2] zero counters of the in-kernel reductions
    double2 *partials_c;
    double *partials_r;
    double *cols;      // per Arnoldi step of a cycle: COL_STRIDE doubles (see col_* below)
    double *host;      // pinned, 2 * 2 * (m + 1) + 8 doubles
    double *host_cols; // pinned, DST_MAX_VEC * COL_STRIDE doubles
    void *dev_base;
    // flexible GMRES (preconditioned mixed solve): the preconditioned directions
    // z_j (m FP32 vectors), two FP32 vectors for the second sweep, the sweep's scratch
    float2 *Z, *pr, *pz2;
    void *sweep_scratch;
};

// One Arnoldi step's record in Workspace::cols: first-pass coefficients
// (DST_MAX_VEC complex), second-pass coefficients (DST_MAX_VEC complex), and
// 8 doubles: [0] ||w||^2 after the last pass, [3] before the first update,
// [6] 1 if the second pass ran, [7] 1 if a bulk-copy wait of the projection or update timed out.
constexpr int COL_STRIDE = 4 * DST_MAX_VEC + 8;

// FP32-stored bases of at least this many unknowns use the bulk-copy fed
// projection and update (measured on the 2+1 workload, 1.77M unknowns: solve
// 0.196 -> 0.183 s against the register-fed kernels).
constexpr int64_t TMA_MIN_UNKNOWNS = 1000000;

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

int setup_workspace(dst_mesh *mesh, int m, bool mixed, Workspace &w, int precond = 0, size_t sweep_bytes = 0) {
    const int64_t n = mesh->n_unknowns;
    const int nblk = DST_MAX_RED_BLOCKS;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
    const size_t oV = take(sizeof(double2) * (size_t)n * (m + 1));
    const size_t ob = take(sizeof(double2) * n);
    const size_t ot = take(sizeof(double2) * n);
    const size_t od = mixed ? take(sizeof(double2) * n) : 0;
    const size_t or64 = mixed ? take(sizeof(double2) * n) : 0;
    const size_t orin = mixed ? take(sizeof(double2) * n) : 0;
    const size_t ox32 = mixed ? take(sizeof(float2) * n) : 0;
    const size_t oy32 = mixed ? take(sizeof(float2) * n) : 0;
    const size_t oh1 = take(sizeof(double2) * DST_MAX_VEC);
    const size_t oh2 = take(sizeof(double2) * DST_MAX_VEC);
    const size_t onrm = take(sizeof(double) * 8);
    const size_t otk = take(sizeof(unsigned) * 8);
    const size_t opc = take(sizeof(double2) * (size_t)nblk * DST_MAX_VEC);
    const size_t opr = take(sizeof(double) * (size_t)nblk);
    const size_t ocols = take(sizeof(double) * (size_t)COL_STRIDE * DST_MAX_VEC);
    const size_t oZ = precond ? take(sizeof(float2) * (size_t)n * m) : 0;
    const bool need_pr = precond == DST_PRECOND_CN_SWEEP2 || precond == DST_PRECOND_CN_LEARNED;
    const size_t opres = need_pr ? take(sizeof(float2) * (size_t)n) : 0;
    const size_t opz2 = precond == DST_PRECOND_CN_SWEEP2 ? take(sizeof(float2) * (size_t)n) : 0;
    const size_t osw = precond ? take(sweep_bytes) : 0;
    const size_t total = off;
    if (mesh->ws_bytes < total) {
        cudaFree(mesh->ws);
        mesh->ws = nullptr;
        mesh->ws_bytes = 0;
        if (dst_internal_injected_alloc_failure()) {
            dst_internal_set_error_detail("dst_solve: workspace allocation failed (injected by dst_testing_set)");
            return DST_ERR_OOM;
        }
        if (cudaMalloc(&mesh->ws, total) != cudaSuccess) {
            mesh->ws = nullptr;
            cudaGetLastError();
            return DST_ERR_OOM;
        }
        mesh->ws_bytes = total;
    }
    char *base = (char *)mesh->ws;
    w.n = n;
    w.m = m;
    w.mixed = mixed;
    w.dev_base = base;
    w.V = (double2 *)(base + oV);
    w.b = (double2 *)(base + ob);
    w.tmp = (double2 *)(base + ot);
    w.d = mixed ? (double2 *)(base + od) : nullptr;
    w.r64 = mixed ? (double2 *)(base + or64) : nullptr;
    w.rin = mixed ? (double2 *)(base + orin) : nullptr;
    w.x32 = mixed ? (float2 *)(base + ox32) : nullptr;
    w.y32 = mixed ? (float2 *)(base + oy32) : nullptr;
    w.h1 = (double2 *)(base + oh1);
    w.h2 = (double2 *)(base + oh2);
    w.nrm = (double *)(base + onrm);
    w.tickets = (unsigned *)(base + otk);
    w.partials_c = (double2 *)(base + opc);
    w.partials_r = (double *)(base + opr);
    w.cols = (double *)(base + ocols);
    w.Z = precond ? (float2 *)(base + oZ) : nullptr;
    w.pr = need_pr ? (float2 *)(base + opres) : nullptr;
    w.pz2 = precond == DST_PRECOND_CN_SWEEP2 ? (float2 *)(base + opz2) : nullptr;
    w.sweep_scratch = precond ? (void *)(base + osw) : nullptr;
    return DST_OK;
}

// Kernel classes reported in dst_solve_stats (index = DST_K_* in diracst.h).
enum { K_APPLY64 = 0, K_APPLY32, K_CAST, K_PROJECT, K_UPDATE, K_SCALE, K_MISC, K_RHS, K_PRECOND, K_NCLASS };

// Per-class accounting of launches, algorithmic bytes / flops and, when
// profiling, device time from CUDA events recorded around each launch on the
// solver's stream (harvested at the solver's host synchronisation points).
// Inside a chain of launches with nothing else enqueued between them (the
// steps of a cycle) one event marks both the end of a launch and the start of
// the next, half the events of separate brackets.
struct Prof {
    bool on = false;
    bool chain = false;      // the previous launch's end event may open the next one
    bool capturing = false;  // recording into a stream capture: events become graph nodes
    double ms[K_NCLASS] = {}, launches[K_NCLASS] = {}, bytes[K_NCLASS] = {}, flops[K_NCLASS] = {};
    struct Pending { int cls; int a, b; };     // indices into line
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> line;             // events recorded since the last harvest
    std::vector<cudaEvent_t> pool;
    int last = -1;                             // line index of the previous launch's end
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    int mark(cudaStream_t s) {
        cudaEvent_t e = get();
        if (capturing) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
        line.push_back(e);
        return (int)line.size() - 1;
    }
    void harvest() {
        for (auto &p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, line[p.a], line[p.b]) == cudaSuccess) ms[p.cls] += t;
            else cudaGetLastError();
        }
        for (auto e : line) pool.push_back(e);
        line.clear();
        pending.clear();
        last = -1;
    }
    ~Prof() {
        for (auto e : line) pool.push_back(e);
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Hessenberg matrix of one GMRES cycle reduced by complex Givens rotations
// [[c, s], [-conj(s), c]] as columns arrive; g holds the rotated right-hand
// side beta e_1, |g_{j+1}| the least-squares residual of the cycle.
struct Hess {
    int m;
    std::vector<cplx> H, g, sn;
    std::vector<double> cs;
    explicit Hess(int m_) : m(m_), H((size_t)(m_ + 1) * m_), g(m_ + 1), sn(m_), cs(m_) {}
    cplx &at(int i, int j) { return H[(size_t)i * m + j]; }
    void start(double beta) {
        std::fill(H.begin(), H.end(), cplx(0.0));
        std::fill(g.begin(), g.end(), cplx(0.0));
        g[0] = beta;
    }
    // column j: h[0..j] and h_{j+1,j} = hn; returns |g_{j+1}|
    double add_column(int j, const cplx *h, double hn) {
        for (int i = 0; i <= j; ++i) at(i, j) = h[i];
        at(j + 1, j) = hn;
        for (int i = 0; i < j; ++i) {
            const cplx t = cs[i] * at(i, j) + sn[i] * at(i + 1, j);
            at(i + 1, j) = -std::conj(sn[i]) * at(i, j) + cs[i] * at(i + 1, j);
            at(i, j) = t;
        }
        const cplx a = at(j, j), b = at(j + 1, j);
        if (std::abs(b) == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
        else if (std::abs(a) == 0.0) { cs[j] = 0.0; sn[j] = 1.0; }
        else {
            const double rho = std::sqrt(std::norm(a) + std::norm(b));
            cs[j] = std::abs(a) / rho;
            sn[j] = (a / std::abs(a)) * std::conj(b) / rho;
        }
        at(j, j) = cs[j] * a + sn[j] * b;
        at(j + 1, j) = 0.0;
        g[j + 1] = -std::conj(sn[j]) * g[j];
        g[j] = cs[j] * g[j];
        return std::abs(g[j + 1]);
    }
    // y = R(0:k,0:k)^{-1} g(0:k) by back substitution, written as sign * y
    // (interleaved re, im) into out.
    void solve(int k, double *out, double sign) {
        std::vector<cplx> y(k);
        for (int i = k - 1; i >= 0; --i) {
            cplx acc = g[i];
            for (int l = i + 1; l < k; ++l) acc -= at(i, l) * y[l];
            y[i] = acc / at(i, i);
        }
        for (int i = 0; i < k; ++i) {
            out[2 * i] = sign * y[i].real();
            out[2 * i + 1] = sign * y[i].imag();
        }
    }
};

struct Solver;

// The captured CUDA graph of one full mixed GMRES cycle (see Solver::enqueue_cycle):
// the executable graph, the per-class accounting one replay adds, and, when
// profiling, the event pairs recorded inside the graph.
struct CycleGraph {
    bool ok = true;                      // false after a failed capture: launch directly
    cudaGraphExec_t exec = nullptr;
    double launches[K_NCLASS] = {}, bytes[K_NCLASS] = {}, flops[K_NCLASS] = {};
    double total_bytes = 0.0;
    std::vector<Prof::Pending> pending;  // indices into events
    std::vector<cudaEvent_t> events;
    int capture(Solver &sv, int steps, bool vlo);
    void account(Solver &sv);
    void harvest(Prof &p) {
        for (auto &q : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, events[q.a], events[q.b]) == cudaSuccess) p.ms[q.cls] += t;
            else cudaGetLastError();
        }
    }
    ~CycleGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto e : events) cudaEventDestroy(e);
    }
};

struct Solver {
    dst_mesh *mesh;
    cudaStream_t s;
    Workspace w;
    int nblk;         // CTAs of the reduction / update passes
    int nblk_proj;    // CTAs of the df32 projection (fewer, longer slices)
    double bytes = 0.0;
    int iters = 0;
    int restarts = 0;
    int reorths = 0;
    int ortho = 0;           // 0: DGKS selective second pass, 1: always two passes, 2: one pass
    int precond = 0;         // DST_PRECOND_*: flexible GMRES with the Crank-Nicolson sweep
    SweepPlan plan;
    double resid_est = 0.0;
    Prof prof;
    CycleGraph graph;

    // Run one launcher (nk kernels) of class cls with its algorithmic bytes / flops.
    template <typename F>
    int run(int cls, int nk, double nbytes, double nflops, F &&launch) {
        int a = -1;
        if (prof.on) a = prof.chain && prof.last >= 0 ? prof.last : prof.mark(s);
        int rc = launch();
        if (prof.on) {
            const int b = prof.mark(s);
            prof.pending.push_back({cls, a, b});
            prof.last = b;
        }
        prof.launches[cls] += nk;
        prof.bytes[cls] += nbytes;
        prof.flops[cls] += nflops;
        bytes += nbytes;
        return rc;
    }

    // out = A in, FP64 or FP32 arithmetic
    int apply(int prec, const double2 *in, double2 *out) {
        const double n = (double)w.n;
        if (prec == DST_FP64)
            return run(K_APPLY64, 1, 32.0 * n, dst_internal_apply_flops(mesh),
                       [&] { return dst_internal_apply(mesh, DST_FP64, in, out, s); });
        int rc = run(K_CAST, 1, 24.0 * n, 0.0, [&] { return dst_k_cast_64_32(w.n, in, w.x32, s); });
        if (rc) return rc;
        rc = run(K_APPLY32, 1, 16.0 * n, dst_internal_apply_flops(mesh),
                 [&] { return dst_internal_apply(mesh, DST_FP32, w.x32, w.y32, s); });
        if (rc) return rc;
        return run(K_CAST, 1, 24.0 * n, 0.0, [&] { return dst_k_cast_32_64(w.n, w.y32, out, s); });
    }
    // gate: second-pass kernels that skip themselves on the device when the
    // DGKS test (nrm[0] < nrm[3] / 2) fails; their bytes are counted only if
    // they ran (second_pass_ran() after the step's synchronisation).
    int project(int nv, const double2 *wv, double2 *h, double *wnrm2 = nullptr, const double *gate = nullptr) {
        const double n = (double)w.n;
        return run(K_PROJECT, wnrm2 ? 3 : 2, gate ? 0.0 : 16.0 * n * (nv + 1),
                   gate ? 0.0 : 8.0 * n * nv + (wnrm2 ? 4.0 * n : 0.0),
                   [&] { return dst_k_project(w.n, nv, w.V, wv, h, w.partials_c, nblk, s, wnrm2, w.partials_r, gate); });
    }
    // second: the step's second Gram-Schmidt pass (bumps the device counter nrm[6] when it runs)
    int update(int nv, const double2 *h, double2 *x, double *nrm2, const double *gate = nullptr, bool second = false) {
        const double n = (double)w.n;
        return run(K_UPDATE, nrm2 ? 2 : 1, gate ? 0.0 : 16.0 * n * (nv + 2),
                   gate ? 0.0 : 8.0 * n * nv + (nrm2 ? 4.0 * n : 0.0),
                   [&] { return dst_k_update(w.n, nv, w.V, h, x, nrm2, w.partials_r, nblk, s, gate,
                                             second ? w.nrm + 6 : nullptr); });
    }
    // account a gated second pass over nv basis vectors that did run
    // bytes of a second Gram-Schmidt pass that ran (vb: bytes per stored entry)
    void count_second_pass(int nv, double vb = 16.0) {
        const double n = (double)w.n;
        const double pb = vb * n * (nv + 1);
        const double ub = vb * n * (nv + 2);
        prof.bytes[K_PROJECT] += pb; prof.flops[K_PROJECT] += 8.0 * n * nv;
        prof.bytes[K_UPDATE] += ub; prof.flops[K_UPDATE] += 8.0 * n * nv;
        bytes += pb + ub;
    }
    int scale(double2 *v) {
        return run(K_SCALE, 1, 32.0 * w.n, 2.0 * w.n, [&] { return dst_k_scale(w.n, v, v, w.nrm, 0.0, s); });
    }
    int residual(const double2 *rhs, const double2 *y, double2 *r, double *nrm2) {
        return run(K_MISC, 2, 48.0 * w.n, 6.0 * w.n,
                   [&] { return dst_k_residual(w.n, rhs, y, r, nrm2, w.partials_r, nblk, s); });
    }

    int read_host(const void *src, size_t bytes_, double *dst) {
        DST_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes_, cudaMemcpyDeviceToHost, s));
        return DST_OK;
    }

    int sync() {
        DST_CUDA_TRY(cudaStreamSynchronize(s));
        if (prof.on) prof.harvest();
        return DST_OK;
    }

    // ||v||^2 into w.nrm[slot] (device), then the value on the host.
    int norm(const double2 *v, int slot, double &out) {
        int rc = run(K_MISC, 2, 16.0 * w.n, 4.0 * w.n,
                     [&] { return dst_k_nrm2(w.n, v, w.nrm + slot, w.partials_r, nblk, s); });
        if (rc) return rc;
        if ((rc = read_host(w.nrm + slot, sizeof(double), w.host)) || (rc = sync())) return rc;
        out = std::sqrt(w.host[0]);
        return DST_OK;
    }

    // V[0] = rhs - A x and beta = ||V[0]|| (x_zero: V[0] = rhs).
    int initial_residual(int prec, const double2 *x, const double2 *rhs, bool x_zero, double &beta) {
        int rc;
        if (x_zero) {
            DST_CUDA_TRY(cudaMemcpyAsync(w.V, rhs, sizeof(double2) * w.n, cudaMemcpyDeviceToDevice, s));
            bytes += 32.0 * w.n;
            return norm(w.V, 0, beta);
        }
        if ((rc = apply(prec, x, w.tmp))) return rc;
        if ((rc = residual(rhs, w.tmp, w.V, w.nrm))) return rc;
        if ((rc = read_host(w.nrm, sizeof(double), w.host)) || (rc = sync())) return rc;
        beta = std::sqrt(w.host[0]);
        return DST_OK;
    }

    // One host synchronisation per Arnoldi step: both Gram-Schmidt columns and
    // the norms / second-pass counter (nrm[0..7]) come back together.
    double reorth_seen = 0.0;
    bool last_second = false;
    int read_step(int nv) {
        DST_CUDA_TRY(cudaMemcpyAsync(w.host, w.h1, sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
        DST_CUDA_TRY(cudaMemcpyAsync(w.host + 2 * DST_MAX_VEC, w.h2, sizeof(double2) * nv, cudaMemcpyDeviceToHost, s));
        DST_CUDA_TRY(cudaMemcpyAsync(w.host + 4 * DST_MAX_VEC, w.nrm, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        int rc = sync();
        if (rc) return rc;
        const double cnt = w.host[4 * DST_MAX_VEC + 6];
        last_second = cnt > reorth_seen;
        reorth_seen = cnt;
        if (last_second) ++reorths;
        return DST_OK;
    }
    bool second_pass_ran() const { return last_second; }

    // Hessenberg column j from the host buffer (first pass at host[0], second
    // pass at host[2*MAXVEC], new norm^2 at host[4*MAXVEC]) into hs; returns
    // DST_ERR_NAN on a non-finite column.
    int take_column(Hess &hs, int j, const double *c1, const double *c2, double hn2, bool &breakdown) {
        const int nv = j + 1;
        std::vector<cplx> col(nv);
        for (int i = 0; i < nv; ++i) col[i] = cplx(c1[2 * i] + c2[2 * i], c1[2 * i + 1] + c2[2 * i + 1]);
        double colsq = 0.0;
        for (auto &c : col) colsq += std::norm(c);
        if (!std::isfinite(hn2) || !std::isfinite(colsq)) return DST_ERR_NAN;
        resid_est = hs.add_column(j, col.data(), std::sqrt(hn2));
        breakdown = std::sqrt(hn2) <= 1e-14 * std::sqrt(colsq + hn2);
        return DST_OK;
    }
    int take_column(Hess &hs, int j, bool &breakdown) {
        const int nv = j + 1;
        std::vector<cplx> col(nv);
        for (int i = 0; i < nv; ++i)
            col[i] = cplx(w.host[2 * i] + w.host[2 * DST_MAX_VEC + 2 * i],
                          w.host[2 * i + 1] + w.host[2 * DST_MAX_VEC + 2 * i + 1]);
        const double hn2 = w.host[4 * DST_MAX_VEC];
        double colsq = 0.0;
        for (auto &c : col) colsq += std::norm(c);
        if (!std::isfinite(hn2) || !std::isfinite(colsq)) return DST_ERR_NAN;
        resid_est = hs.add_column(j, col.data(), std::sqrt(hn2));
        breakdown = std::sqrt(hn2) <= 1e-14 * std::sqrt(colsq + hn2);
        return DST_OK;
    }

    // Restarted GMRES(m) on A_prec x = rhs, FP64 basis and FP64 Gram-Schmidt,
    // until ||rhs - A x|| <= tol_abs, max_iters Arnoldi steps in total
    // (this->iters) or max_cycles cycles; in the last case the caller computes
    // the residual (beta_out = -1).
    int gmres(int prec, double2 *x, const double2 *rhs, bool x_zero, double tol_abs, int max_iters,
              double &beta_out, int max_cycles = 0x7fffffff) {
        if (ortho == 2) DST_CUDA_TRY(cudaMemsetAsync(w.h2, 0, sizeof(double2) * DST_MAX_VEC, s));
        const int m = w.m;
        const int64_t n = w.n;
        double beta;
        int rc = initial_residual(prec, x, rhs, x_zero, beta);
        if (rc) return rc;
        if (!std::isfinite(beta)) return DST_ERR_NAN;
        Hess hs(m);
        bool breakdown = false;
        int cycles = 0;
        while (beta > tol_abs && iters < max_iters && !breakdown) {
            if ((rc = scale(w.V))) return rc;   // V0 = r / beta
            hs.start(beta);
            int k = 0;
            for (int j = 0; j < m; ++j) {
                double2 *vj = w.V + (size_t)j * n;
                double2 *wv = w.V + (size_t)(j + 1) * n;
                if ((rc = apply(prec, vj, wv))) return rc;
                const int nv = j + 1;
                // classical Gram-Schmidt pass; ||A v_j||^2 (before) into nrm[3], ||w||^2 (after) into nrm[0]
                if ((rc = project(nv, wv, w.h1, w.nrm + 3))) return rc;
                if ((rc = update(nv, w.h1, wv, w.nrm))) return rc;
                // second pass, gated on the device by the DGKS test unless always on
                // (CGS2) or never (ortho 2: w.h2 stays zero)
                const double *gate = ortho == 1 ? nullptr : w.nrm;
                if (ortho != 2) {
                    if ((rc = project(nv, wv, w.h2, nullptr, gate))) return rc;
                    if ((rc = update(nv, w.h2, wv, w.nrm, gate, true))) return rc;
                }
                if ((rc = scale(wv))) return rc;     // normalise on the device (1/sqrt(nrm))
                if ((rc = read_step(nv))) return rc;
                if (second_pass_ran() && gate) count_second_pass(nv);
                ++iters;
                if ((rc = take_column(hs, j, breakdown))) return rc;
                k = j + 1;
                if (breakdown || resid_est <= tol_abs || iters >= max_iters) break;
            }
            // x += V y  (update with h = -y)
            hs.solve(k, w.host, -1.0);
            DST_CUDA_TRY(cudaMemcpyAsync(w.h1, w.host, sizeof(double2) * k, cudaMemcpyHostToDevice, s));
            if ((rc = update(k, w.h1, x, nullptr))) return rc;
            ++restarts;
            if (++cycles >= max_cycles) {
                beta_out = -1.0;
                return DST_OK;
            }
            if ((rc = initial_residual(prec, x, rhs, false, beta))) return rc;
            if (!std::isfinite(beta)) return DST_ERR_NAN;
        }
        beta_out = beta;
        return DST_OK;
    }

    // BiCGSTAB (van der Vorst 1992) in FP64: two operator applies and four inner
    // products per step; the scalars alpha, beta, omega stay on the device, so a
    // step needs one host synchronisation (the residual norm for the stop test).
    int bicgstab(double2 *x, const double2 *rhs, bool x_zero, double tol_abs, int max_iters, double &beta_out) {
        const int64_t n = w.n;
        const double dn = (double)n;
        double2 *rhat = w.V, *r = w.V + n, *pv = w.V + 2 * n, *v = w.V + 3 * n, *sv = w.V + 4 * n, *t = w.V + 5 * n;
        double2 *sc = w.h2;
        auto dot = [&](const double2 *a, const double2 *bb, double2 *out) {
            return run(K_PROJECT, 2, 32.0 * dn, 8.0 * dn,
                       [&] { return dst_k_project(n, 1, a, bb, out, w.partials_c, nblk, s); });
        };
        double beta;
        int rc = initial_residual(DST_FP64, x, rhs, x_zero, beta);       // V[0] = rhs - A x
        if (rc) return rc;
        if (!std::isfinite(beta)) return DST_ERR_NAN;
        // The recursively updated residual drifts from rhs - A x; when it meets the
        // tolerance but the true residual does not, the method restarts from x
        // with the true residual as its new shadow vector.
        while (beta > tol_abs && iters < max_iters) {
            ++restarts;
            DST_CUDA_TRY(cudaMemcpyAsync(r, rhat, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
            DST_CUDA_TRY(cudaMemsetAsync(pv, 0, sizeof(double2) * n, s));
            DST_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(double2) * n, s));
            if ((rc = dst_k_bicg_scalar(3, sc, s))) return rc;
            double rn = beta;
            while (rn > tol_abs && iters < max_iters) {
                if ((rc = dot(rhat, r, sc + 7))) return rc;                             // rho_new = (rhat, r)
                if ((rc = dst_k_bicg_scalar(0, sc, s))) return rc;                      // beta, rho
                if ((rc = run(K_MISC, 1, 64.0 * dn, 12.0 * dn, [&] { return dst_k_bicg_p(n, r, v, pv, sc, s); })))
                    return rc;
                if ((rc = apply(DST_FP64, pv, v))) return rc;                           // v = A p
                if ((rc = dot(rhat, v, sc + 4))) return rc;
                if ((rc = dst_k_bicg_scalar(1, sc, s))) return rc;                      // alpha
                if ((rc = run(K_MISC, 1, 48.0 * dn, 8.0 * dn, [&] { return dst_k_bicg_s(n, r, v, sv, sc, s); })))
                    return rc;
                if ((rc = apply(DST_FP64, sv, t))) return rc;                           // t = A s
                if ((rc = dot(t, sv, sc + 5))) return rc;
                if ((rc = run(K_MISC, 2, 16.0 * dn, 4.0 * dn, [&] {
                         return dst_k_nrm2(n, t, reinterpret_cast<double *>(sc + 6), w.partials_r, nblk, s);
                     })))
                    return rc;
                if ((rc = dst_k_bicg_scalar(2, sc, s))) return rc;                      // omega
                if ((rc = run(K_MISC, 2, 96.0 * dn, 24.0 * dn,
                              [&] { return dst_k_bicg_xr(n, x, pv, sv, t, r, sc, w.nrm, w.partials_r, nblk, s); })))
                    return rc;
                DST_CUDA_TRY(cudaMemcpyAsync(w.host, w.nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
                if ((rc = sync())) return rc;
                ++iters;
                rn = std::sqrt(w.host[0]);
                resid_est = rn;
                if (!std::isfinite(rn)) return DST_ERR_NAN;
            }
            if ((rc = initial_residual(DST_FP64, x, rhs, false, beta))) return rc;   // true residual
            if (!std::isfinite(beta)) return DST_ERR_NAN;
        }
        beta_out = beta;
        return DST_OK;
    }

    // z = M(v) with the Crank-Nicolson sweep; the second variant adds M(v - A M(v)),
    // the learned one a correction computed from rho = v - A M(v); tmp is a free
    // FP32 vector (the next basis slot), holding A M(v) and then scratch.
    int precondition(const float2 *v, float2 *z, float2 *tmp) {
        const int64_t n = w.n;
        const double dn = (double)n;
        if (precond == DST_PRECOND_BLOCK_JACOBI)       // z = blockdiag(A_nn)^-1 v
            return run(K_PRECOND, 1, (16.0 + 8.0 * mesh->nc) * dn, 8.0 * mesh->nc * dn,
                       [&] { return dst_internal_jacobi_apply(mesh, v, z, s); });
        const double sweep_bytes = (plan.has_fft ? 48.0 : 40.0) * dn + (double)plan.table_bytes * plan.g.nt;
        int rc = run(K_PRECOND, plan.has_fft ? 4 : 3, sweep_bytes, 0.0,
                     [&] { return dst_sweep_apply(plan, n, v, z, s); });
        if (rc || precond == DST_PRECOND_CN_SWEEP) return rc;
        if ((rc = run(K_APPLY32, 1, 16.0 * dn, dst_internal_apply_flops(mesh),
                      [&] { return dst_internal_apply(mesh, DST_FP32, z, tmp, s); })))
            return rc;
        if ((rc = run(K_MISC, 1, 24.0 * dn, 2.0 * dn, [&] { return dst_k_sub_f32(n, v, tmp, w.pr, s); }))) return rc;
        if (precond == DST_PRECOND_CN_LEARNED) {      // z += alpha U(rho / ||rho||), rho = v - A M_CN(v)
            int nk = 0;
            rc = run(K_PRECOND, 0, 0.0, 0.0,
                     [&] { return dst_internal_unet_correct(mesh->unet, mesh, w.pr, z, tmp, s, &nk); });
            prof.launches[K_PRECOND] += nk;
            return rc;
        }
        if ((rc = run(K_PRECOND, plan.has_fft ? 4 : 3, sweep_bytes, 0.0,
                      [&] { return dst_sweep_apply(plan, n, w.pr, w.pz2, s); })))
            return rc;
        return run(K_MISC, 1, 24.0 * dn, 2.0 * dn, [&] { return dst_k_add_f32(n, w.pz2, z, s); });
    }

    // The Arnoldi steps of one mixed cycle: a zeroed record per step, then per
    // step the FP32 apply, both Gram-Schmidt passes (the second gated on the
    // device) and the scaling, all on stream s.
    int enqueue_steps(int steps, bool vlo) {
        const int64_t n = w.n;
        // large FP32-stored bases: the projection and the update fed by bulk asynchronous copies
        const bool use_tma = !vlo && n >= TMA_MIN_UNKNOWNS;
        const int nblk_tma = dst_tma_projection_blocks(n);
        const double dn = (double)n;
        const double vb = vlo ? 16.0 : 8.0;
        const int64_t vs = (vlo ? 2 : 1) * n;
        float2 *Vd = reinterpret_cast<float2 *>(w.V);
        int rc;
        DST_CUDA_TRY(cudaMemsetAsync(w.cols, 0, sizeof(double) * COL_STRIDE * steps, s));
        prof.chain = true;          // only kernels are enqueued until the loop ends
        prof.last = -1;
        for (int j = 0; j < steps; ++j) {
            float2 *vj = Vd + (size_t)j * vs;
            float2 *wv = Vd + (size_t)(j + 1) * vs;
            const int nv = j + 1;
            double2 *c1 = reinterpret_cast<double2 *>(w.cols + (size_t)j * COL_STRIDE);
            double2 *c2 = c1 + DST_MAX_VEC;
            double *nr = w.cols + (size_t)j * COL_STRIDE + 4 * DST_MAX_VEC;
            // flexible GMRES: the operator is applied to z_j = M(v_j), kept in Z
            const float2 *av = vj;
            if (precond) {
                float2 *zj = w.Z + (size_t)j * n;
                if ((rc = precondition(vj, zj, wv))) return rc;
                av = zj;
            }
            // FP32 apply straight from the hi plane of v_j (or z_j) into the hi plane of w
            if ((rc = run(K_APPLY32, 1, 16.0 * dn, dst_internal_apply_flops(mesh),
                          [&] { return dst_internal_apply(mesh, DST_FP32, av, wv, s); })))
                return rc;
            if ((rc = run(K_PROJECT, 1, vb * dn * nv + 8.0 * dn, 8.0 * dn * nv, [&] {
                     return use_tma ? dst_k_project_tma(n, nv, Vd, wv, c1, w.partials_c, nblk_tma, s, nr + 3, nullptr,
                                                        w.tickets, nr + 7)
                                    : dst_k_project_df(n, nv, Vd, wv, true, c1, w.partials_c, nblk_proj, s, nr + 3,
                                                       w.partials_r, nullptr, w.tickets, vlo);
                 })))
                return rc;
            if ((rc = run(K_UPDATE, 1, vb * dn * nv + 8.0 * dn + vb * dn, 8.0 * dn * nv, [&] {
                     return use_tma ? dst_k_update_tma(n, nv, Vd, c1, wv, nr, w.partials_r, nblk_tma, s, nullptr,
                                                       nullptr, w.tickets + 1, nr + 7)
                                    : dst_k_update_df(n, nv, Vd, c1, wv, true, nr, w.partials_r, nblk, s, nullptr,
                                                      nullptr, w.tickets + 1, vlo);
                 })))
                return rc;
            // second pass, gated on the device by the DGKS test unless always on
            // (CGS2) or never (ortho 2: the record's second-pass slots stay zero)
            const double *gate = ortho == 1 ? nullptr : nr;
            const double g2 = gate ? 0.0 : 1.0;
            if (ortho != 2 && (rc = run(K_PROJECT, 1, g2 * vb * dn * (nv + 1), g2 * 8.0 * dn * nv, [&] {
                     return use_tma ? dst_k_project_tma(n, nv, Vd, wv, c2, w.partials_c, nblk_tma, s, nullptr, gate,
                                                        w.tickets, nr + 7)
                                    : dst_k_project_df(n, nv, Vd, wv, !vlo, c2, w.partials_c, nblk_proj, s, nullptr,
                                                       nullptr, gate, w.tickets, vlo);
                 })))
                return rc;
            if (ortho != 2 && (rc = run(K_UPDATE, 1, g2 * vb * dn * (nv + 2), g2 * 8.0 * dn * nv, [&] {
                     return use_tma ? dst_k_update_tma(n, nv, Vd, c2, wv, nr, w.partials_r, nblk_tma, s, gate, nr + 6,
                                                       w.tickets + 1, nr + 7)
                                    : dst_k_update_df(n, nv, Vd, c2, wv, !vlo, nr, w.partials_r, nblk, s, gate,
                                                      nr + 6, w.tickets + 1, vlo);
                 })))
                return rc;
            if ((rc = run(K_SCALE, 1, 2.0 * vb * dn, 6.0 * dn, [&] { return dst_k_scale_df(n, wv, nr, s, vlo); })))
                return rc;
        }
        prof.chain = false;
        return DST_OK;
    }

    // Enqueue a cycle's steps; a full cycle (steps == m) is captured once as a
    // CUDA graph and replayed afterwards: same launches, same arguments, one
    // graph launch instead of ~6 m kernel launches.  Falls back to direct
    // launches if capture is not possible.
    int full_cycles = 0;     // full cycles enqueued so far (the first runs uncaptured)
    int enqueue_cycle(int steps, bool full, bool vlo, bool &replayed) {
        replayed = false;
        // capture from the second full cycle on: by then every kernel of the
        // cycle has been launched once (per-device attributes set outside capture)
        if (full && graph.ok && !graph.exec && full_cycles > 0) {
            int rc = graph.capture(*this, steps, vlo);
            if (rc) return rc;
        }
        if (full) ++full_cycles;
        if (full && graph.exec) {
            DST_CUDA_TRY(cudaGraphLaunch(graph.exec, s));
            graph.account(*this);
            replayed = true;
            return DST_OK;
        }
        return enqueue_steps(steps, vlo);
    }

    // One GMRES(m) cycle for the correction equation A d = r (d = 0 on entry),
    // FP32 operator apply on a df32 basis with df32 Gram-Schmidt: V_0 = r/||r||
    // (||r||^2 in w.nrm[rslot]), d += V y at the end (FP64).
    // vlo = false: the basis is stored in FP32 (hi planes only, 8 B per entry)
    // and the same compensated kernels run on it.
    int cycle_df(double2 *d, const double2 *r, int rslot, double rnorm, double tol_abs, int max_iters, bool vlo) {
        NvtxRange range("GMRES cycle");
        const int m = w.m;
        const int64_t n = w.n;
        const double dn = (double)n;
        const double vb = vlo ? 16.0 : 8.0;             // bytes per stored basis entry
        float2 *Vd = reinterpret_cast<float2 *>(w.V);   // (m+1) vectors
        int rc = run(K_SCALE, 1, 16.0 * dn + vb * dn, 2.0 * dn,
                     [&] { return dst_k_split_f64_df(n, r, w.nrm + rslot, Vd, s, vlo); });
        if (rc) return rc;
        Hess hs(m);
        hs.start(rnorm);
        // Every step of the cycle runs on the device (the second pass is gated
        // there, norms and scaling too), so all steps are enqueued at once, each
        // writing its own record in w.cols; the columns come back with one
        // synchronisation per cycle.  Steps after the one that meets the
        // tolerance (or breaks down) have run but are discarded.
        const int steps = std::min(m, max_iters - iters);
        if (steps < 1) return DST_OK;
        bool replayed = false;
        if ((rc = enqueue_cycle(steps, steps == m, vlo, replayed))) return rc;
        DST_CUDA_TRY(cudaMemcpyAsync(w.host_cols, w.cols, sizeof(double) * COL_STRIDE * steps,
                                     cudaMemcpyDeviceToHost, s));
        if ((rc = sync())) return rc;
        if (replayed) graph.harvest(prof);
        bool breakdown = false;
        int k = 0;
        for (int j = 0; j < steps; ++j) {
            const double *c1 = w.host_cols + (size_t)j * COL_STRIDE;
            const double *nr = c1 + 4 * DST_MAX_VEC;
            if (nr[7] != 0.0) {
                dst_internal_set_error_detail("dst_solve: a bulk-copy wait of the Gram-Schmidt timed out");
                return DST_ERR_CUDA;
            }
            if (nr[6] > 0.0) {
                ++reorths;
                if (ortho != 1) count_second_pass(j + 1, vb);
            }
            ++iters;
            if ((rc = take_column(hs, j, c1, c1 + 2 * DST_MAX_VEC, nr[0], breakdown))) return rc;
            k = j + 1;
            if (breakdown || resid_est <= tol_abs) break;
        }
        hs.solve(k, w.host, 1.0);
        DST_CUDA_TRY(cudaMemcpyAsync(w.h1, w.host, sizeof(double2) * k, cudaMemcpyHostToDevice, s));
        const float2 *basis = precond ? w.Z : Vd;       // flexible GMRES: d = Z y
        // large FP32-stored bases: the basis fed by bulk copies; a failed wait flags nrm[7]
        const bool tma = !vlo && n >= TMA_MIN_UNKNOWNS;
        if ((rc = run(K_UPDATE, 1, vb * dn * k + 32.0 * dn, 8.0 * dn * k, [&] {
                 return tma ? dst_k_combine_tma(n, k, basis, w.h1, d, dst_tma_projection_blocks(n), s, w.nrm + 7)
                            : dst_k_combine_df(n, k, basis, w.h1, d, s, vlo);
             })))
            return rc;
        ++restarts;
        return DST_OK;
    }
};

// A private stream per thread for capturing (the caller's stream may be the
// legacy default stream, which cannot be captured).  It is destroyed when its
// thread exits, so that short-lived threads (the batch call's workers) leave no
// streams behind.
struct ThreadCaptureStream {
    cudaStream_t s = nullptr;
    int dev = -1;
    void release() {
        if (!s) return;
        int prev = -1;
        const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
        cudaSetDevice(dev);
        cudaStreamDestroy(s);
        if (have_prev) cudaSetDevice(prev);
        cudaGetLastError();
        s = nullptr;
    }
    ~ThreadCaptureStream() { release(); }
};

static cudaStream_t capture_stream() {
    static thread_local ThreadCaptureStream tl;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (!tl.s || tl.dev != dev) {
        tl.release();
        if (cudaStreamCreateWithFlags(&tl.s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            tl.s = nullptr;
            return nullptr;
        }
        tl.dev = dev;
    }
    return tl.s;
}

int CycleGraph::capture(Solver &sv, int steps, bool vlo) {
    cudaStream_t cs = capture_stream();
    if (!cs) { ok = false; return DST_OK; }
    // the accounting of the enqueue is taken as the per-replay amount, not counted now
    Prof &p = sv.prof;
    double l0[K_NCLASS], b0[K_NCLASS], f0[K_NCLASS];
    for (int c = 0; c < K_NCLASS; ++c) { l0[c] = p.launches[c]; b0[c] = p.bytes[c]; f0[c] = p.flops[c]; }
    const double tb0 = sv.bytes;
    const size_t line0 = p.line.size(), pend0 = p.pending.size();
    const int last0 = p.last;
    cudaStream_t saved = sv.s;
    sv.s = cs;
    int rc = DST_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        sv.s = saved;
        ok = false;
        return DST_OK;
    }
    p.capturing = true;
    try {
        rc = sv.enqueue_steps(steps, vlo);
    } catch (...) {
        rc = DST_ERR_OOM;      // a failed host allocation: the capture still ends below
    }
    p.capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    sv.s = saved;
    cudaGraphExec_t ex = nullptr;
    const bool good = rc == DST_OK && ec == cudaSuccess && g &&
                      cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    // events recorded into the graph belong to it
    for (size_t k = line0; k < p.line.size(); ++k) events.push_back(p.line[k]);
    for (size_t k = pend0; k < p.pending.size(); ++k)
        pending.push_back({p.pending[k].cls, p.pending[k].a - (int)line0, p.pending[k].b - (int)line0});
    p.line.resize(line0);
    p.pending.resize(pend0);
    p.last = last0;
    p.chain = false;
    for (int c = 0; c < K_NCLASS; ++c) {
        launches[c] = p.launches[c] - l0[c]; bytes[c] = p.bytes[c] - b0[c]; flops[c] = p.flops[c] - f0[c];
        p.launches[c] = l0[c]; p.bytes[c] = b0[c]; p.flops[c] = f0[c];
    }
    total_bytes = sv.bytes - tb0;
    sv.bytes = tb0;
    if (!good) {
        if (ex) cudaGraphExecDestroy(ex);
        for (auto e : events) cudaEventDestroy(e);
        events.clear();
        pending.clear();
        ok = false;
        return DST_OK;
    }
    exec = ex;
    return DST_OK;
}

void CycleGraph::account(Solver &sv) {
    for (int c = 0; c < K_NCLASS; ++c) {
        sv.prof.launches[c] += launches[c]; sv.prof.bytes[c] += bytes[c]; sv.prof.flops[c] += flops[c];
    }
    sv.bytes += total_bytes;
}

}  // namespace

extern "C" int dst_default_solve_opts(dst_solve_opts *o) {
    if (!o) return DST_ERR_ARG;
    o->restart = 30;
    o->max_iters = 100000;
    o->rtol = 1e-8;
    o->mixed_precision = 0;
    o->inner_rtol = 1e-4;
    o->max_refine = 100000;
    o->inner_cycles = 1;
    o->use_initial_guess = 0;
    o->profile = 0;
    o->ortho = 0;
    o->mixed_ortho = 2;
    o->method = 0;
    o->batch_cta_max = -1;
    o->precond = DST_PRECOND_NONE;
    return DST_OK;
}

static int solve_impl(dst_mesh *mesh, const dst_solve_opts &o, double2 *psi, dst_solve_stats &st,
                      cudaStream_t s) {
    NvtxRange range("dst_solve");
    const bool mixed = o.mixed_precision != 0;
    Solver sv;
    sv.mesh = mesh;
    sv.s = s;
    sv.nblk = dst_reduction_blocks(mesh->n_unknowns);
    // an FP32-stored basis moves half the bytes per entry: slices of 2048
    // entries, at most the 3 CTAs per SM that its projection's registers allow
    sv.nblk_proj = mixed && o.mixed_ortho == 2 ? std::min(dst_reduction_blocks(mesh->n_unknowns), 3 * 152)
                                               : dst_projection_blocks(mesh->n_unknowns);
    sv.ortho = o.ortho;
    sv.precond = o.precond;
    size_t sweep_bytes = 0;
    const bool sweep = o.precond && o.precond != DST_PRECOND_BLOCK_JACOBI;
    if (sweep) {
        int rp = dst_sweep_plan(mesh, sv.plan);
        if (rp) return rp;
        sweep_bytes = dst_sweep_scratch_bytes(sv.plan, mesh->n_unknowns);
    }
    int rc = setup_workspace(mesh, o.method == 1 ? std::max(o.restart, 5) : o.restart, mixed, sv.w, o.precond,
                             sweep_bytes);
    if (rc) return rc;
    if (sweep && (rc = dst_sweep_setup(mesh, sv.plan, sv.w.sweep_scratch, s))) return rc;
    if (o.precond == DST_PRECOND_BLOCK_JACOBI && (rc = dst_internal_jacobi_setup(mesh, s))) return rc;
    // the mesh owns its page-locked record buffer (freed with the mesh), so
    // solves from short-lived threads leave no pinned memory behind
    if (!mesh->host_pinned) {
        const size_t nd = 8 * DST_MAX_VEC + 16 + (size_t)COL_STRIDE * DST_MAX_VEC;
        if (cudaMallocHost(&mesh->host_pinned, sizeof(double) * nd) != cudaSuccess) {
            cudaGetLastError();
            mesh->host_pinned = nullptr;
            return DST_ERR_OOM;
        }
    }
    double *pinned = mesh->host_pinned;
    sv.w.host = pinned;
    sv.w.host_cols = pinned + 8 * DST_MAX_VEC + 16;
    // first solve on this mesh: pick the apply tile shapes (the basis storage,
    // (m + 1) x 16 n bytes, is free scratch at this point)
    if (!mesh->tuned && (rc = dst_internal_tune(mesh, sv.w.V, s))) return rc;
    const int64_t n = mesh->n_unknowns;
    // b = -D_w21 psi0 and ||b||
    sv.prof.on = o.profile != 0;
    DST_CUDA_TRY(cudaMemsetAsync(sv.w.nrm, 0, 8 * sizeof(double), s));      // nrm[7]: the combine's failed-wait flag
    DST_CUDA_TRY(cudaMemsetAsync(sv.w.tickets, 0, 8 * sizeof(unsigned), s));
    if ((rc = sv.run(K_RHS, 1, 16.0 * n + 16.0 * mesh->n_spatial * mesh->nc, 0.0,
                     [&] { return dst_internal_rhs(mesh, sv.w.b, s); })))
        return rc;
    double bnorm;
    if ((rc = sv.norm(sv.w.b, 1, bnorm))) return rc;
    if (!std::isfinite(bnorm)) return DST_ERR_NAN;
    if (!o.use_initial_guess) DST_CUDA_TRY(cudaMemsetAsync(psi, 0, sizeof(double2) * n, s));
    if (bnorm == 0.0) {
        DST_CUDA_TRY(cudaMemsetAsync(psi, 0, sizeof(double2) * n, s));
        DST_CUDA_TRY(cudaStreamSynchronize(s));
        st.rel_resid_true = 0.0;
        st.bytes_moved = sv.bytes;
        return DST_OK;
    }
    const double tol = o.rtol * bnorm;
    double beta = 0.0;
    if (o.method == 1) {
        rc = sv.bicgstab(psi, sv.w.b, !o.use_initial_guess, tol, o.max_iters, beta);
        if (rc) return rc;
    } else if (!mixed) {
        rc = sv.gmres(DST_FP64, psi, sv.w.b, !o.use_initial_guess, tol, o.max_iters, beta);
        if (rc) return rc;
    } else {
        // r64 = b - A64 x
        double rnorm;
        if (!o.use_initial_guess) {
            DST_CUDA_TRY(cudaMemcpyAsync(sv.w.r64, sv.w.b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
            rnorm = bnorm;
        } else {
            if ((rc = sv.apply(DST_FP64, psi, sv.w.tmp))) return rc;
            if ((rc = sv.residual(sv.w.b, sv.w.tmp, sv.w.r64, sv.w.nrm + 2))) return rc;
            DST_CUDA_TRY(cudaMemcpyAsync(sv.w.host, sv.w.nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
            if ((rc = sv.sync())) return rc;
            rnorm = std::sqrt(sv.w.host[0]);
        }
        // df32 / FP32-stored Gram-Schmidt runs each cycle from a correction of 0 on a
        // right-hand side whose norm^2 sits in nrm[2]: the refinement residual r64
        // first, then for further cycles of the same refinement the inner residual
        // r64 - A d with the FP32 operator, the cycle's correction added to d
        const bool use_df = o.mixed_ortho != 1;
        const int cycles = o.inner_cycles > 0 ? o.inner_cycles : 0x7fffffff;
        if (!o.use_initial_guess) {
            DST_CUDA_TRY(cudaMemcpyAsync(sv.w.nrm + 2, sv.w.nrm + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        int refine = 0;
        while (rnorm > tol && refine < o.max_refine && sv.iters < o.max_iters) {
            if (!std::isfinite(rnorm)) return DST_ERR_NAN;
            double inner_beta;
            DST_CUDA_TRY(cudaMemsetAsync(sv.w.d, 0, sizeof(double2) * n, s));
            const double itol = std::max(o.inner_rtol * rnorm, 0.5 * tol);
            if (use_df) {
                rc = sv.cycle_df(sv.w.d, sv.w.r64, 2, rnorm, itol, o.max_iters, o.mixed_ortho == 0);
                for (int c = 1; rc == DST_OK && c < cycles && sv.resid_est > itol && sv.iters < o.max_iters; ++c) {
                    NvtxRange ir("inner residual (FP32)");
                    if ((rc = sv.apply(DST_FP32, sv.w.d, sv.w.tmp))) return rc;
                    if ((rc = sv.residual(sv.w.r64, sv.w.tmp, sv.w.rin, sv.w.nrm + 2))) return rc;
                    DST_CUDA_TRY(cudaMemcpyAsync(sv.w.host, sv.w.nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
                    if ((rc = sv.sync())) return rc;
                    const double rin = std::sqrt(sv.w.host[0]);
                    if (!std::isfinite(rin)) return DST_ERR_NAN;
                    if (rin <= itol) break;
                    rc = sv.cycle_df(sv.w.d, sv.w.rin, 2, rin, itol, o.max_iters, o.mixed_ortho == 0);
                }
            } else
                rc = sv.gmres(DST_FP32, sv.w.d, sv.w.r64, true, itol, o.max_iters, inner_beta,
                              o.inner_cycles > 0 ? o.inner_cycles : 0x7fffffff);
            if (rc) return rc;
            NvtxRange rr("refinement residual (FP64)");
            if ((rc = sv.run(K_MISC, 1, 48.0 * n, 2.0 * n, [&] { return dst_k_axpy1(n, sv.w.d, psi, s); }))) return rc;
            if ((rc = sv.apply(DST_FP64, psi, sv.w.tmp))) return rc;
            if ((rc = sv.residual(sv.w.b, sv.w.tmp, sv.w.r64, sv.w.nrm + 2))) return rc;
            DST_CUDA_TRY(cudaMemcpyAsync(sv.w.host, sv.w.nrm + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
            if ((rc = sv.sync())) return rc;
            rnorm = std::sqrt(sv.w.host[0]);
            ++refine;
        }
        st.refinements = refine;
        beta = rnorm;
    }
    DST_CUDA_TRY(cudaMemcpyAsync(sv.w.host + 1, sv.w.nrm + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((rc = sv.sync())) return rc;
    if (sv.w.host[1] != 0.0) {
        dst_internal_set_error_detail("dst_solve: a bulk-copy wait of the end-of-cycle combine timed out");
        return DST_ERR_CUDA;
    }
    for (int c = 0; c < K_NCLASS; ++c) {
        st.kernel_ms[c] = sv.prof.ms[c];
        st.kernel_launches[c] = sv.prof.launches[c];
        st.kernel_bytes[c] = sv.prof.bytes[c];
        st.kernel_flops[c] = sv.prof.flops[c];
        st.launches += sv.prof.launches[c];
    }
    st.iters = sv.iters;
    st.reorths = sv.reorths;
    st.restarts = sv.restarts;
    st.rel_resid_true = beta / bnorm;
    st.rel_resid_est = sv.resid_est / bnorm;
    st.bytes_moved = sv.bytes;
    if (!std::isfinite(beta)) return DST_ERR_NAN;
    return beta <= tol ? DST_OK : DST_NOT_CONVERGED;
}

extern "C" int dst_solve(dst_mesh *mesh, const dst_solve_opts *opts, void *psi, dst_solve_stats *stats,
                         void *stream) {
    auto t0 = std::chrono::steady_clock::now();
    dst_solve_stats st = {};
    int rc;
    dst_solve_opts o;
    dst_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!mesh || !psi || o.restart < 1 || o.restart > DST_MAX_VEC - 1 || o.max_iters < 0 || !(o.rtol >= 0) ||
        (o.mixed_precision && (!(o.inner_rtol > 0) || o.max_refine < 1)) || o.ortho < 0 || o.ortho > 2 ||
        o.mixed_ortho < 0 || o.mixed_ortho > 2 || o.inner_cycles < 0 || o.method < 0 || o.method > 1 ||
        (o.method == 1 && o.mixed_precision) || o.precond < 0 || o.precond > DST_PRECOND_BLOCK_JACOBI ||
        (o.precond == DST_PRECOND_CN_LEARNED && !dst_internal_unet_fits(mesh->unet, mesh)) ||
        (o.precond && (!o.mixed_precision || o.mixed_ortho != 2 || o.method != 0))) {
        rc = DST_ERR_ARG;
    } else if (!mesh->d_psi0) {
        rc = DST_ERR_STATE;
    } else {
        rc = dst_internal_guard("dst_solve",
                                [&] { return solve_impl(mesh, o, (double2 *)psi, st, (cudaStream_t)stream); });
    }
    st.status = rc;
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = st;
    return rc;
}
