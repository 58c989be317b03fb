// Mesh objects and the C ABI entry points that are not the solver
// (Algorithm 1 steps 1-5: mesh, initial data, operator, right-hand side).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>

#include "internal.h"

static thread_local char g_last_cuda_error[256];

void dst_internal_set_cuda_error(cudaError_t e, const char *expr, const char *file, int line) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s failed at %s:%d: %s", expr, file, line,
             cudaGetErrorString(e));
}

void dst_internal_set_error_detail(const char *msg) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s", msg);
}

void dst_internal_set_exception_detail(const char *call, const char *what) {
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: host allocation or thread start failed: %s", call,
             what);
}

extern "C" const char *dst_last_error_detail(void) { return g_last_cuda_error; }

// Testing hooks: process-wide knobs that make failure paths reachable without
// faulting the GPU (see dst_testing_set in diracst.h).
static std::atomic<long long> g_test_wait_limit{-1};     // -1: the standard limit
static std::atomic<long long> g_test_fail_allocs{0};

unsigned dst_internal_wait_limit(unsigned standard) {
    const long long v = g_test_wait_limit.load();
    return v < 0 ? standard : (unsigned)v;
}

bool dst_internal_injected_alloc_failure() {
    long long v = g_test_fail_allocs.load();
    while (v > 0)
        if (g_test_fail_allocs.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

extern "C" int dst_testing_set(int hook, int64_t value) {
    switch (hook) {
        case DST_TEST_WAIT_LIMIT:
            if (value < -1 || value > 0xffffffffLL) {
                dst_internal_set_error_detail("dst_testing_set: wait limit must be -1 or 0 .. 2^32-1");
                return DST_ERR_ARG;
            }
            g_test_wait_limit.store((long long)value);
            return DST_OK;
        case DST_TEST_FAIL_ALLOC:
            if (value < 0) {
                dst_internal_set_error_detail("dst_testing_set: allocation failure count must be >= 0");
                return DST_ERR_ARG;
            }
            g_test_fail_allocs.store((long long)value);
            return DST_OK;
        default:
            dst_internal_set_error_detail("dst_testing_set: unknown hook");
            return DST_ERR_ARG;
    }
}

extern "C" const char *dst_status_string(int status) {
    switch (status) {
        case DST_OK: return "ok";
        case DST_NOT_CONVERGED: return "not converged (iteration cap reached)";
        case DST_ERR_ARG: return "invalid argument";
        case DST_ERR_OOM: return "out of memory";
        case DST_ERR_CUDA: return "CUDA error";
        case DST_ERR_NAN: return "non-finite value";
        case DST_ERR_STATE: return "missing input (initial data not set)";
        default: return "unknown status";
    }
}

OpParams dst_internal_params(const dst_mesh *mesh) {
    OpParams p;
    for (int k = 0; k < 3; ++k) {
        p.ax[k].n = mesh->nu[k];
        p.ax[k].nel = mesh->nel[k];
        p.ax[k].bc = mesh->bc[k];
        p.ax[k].u0 = mesh->u0[k];
        p.ax[k].h = mesh->h[k];
    }
    p.nt = mesh->nt;
    p.ht = mesh->ht;
    p.m = mesh->m;
    p.vmode = mesh->v_general ? 1 : (mesh->V.empty() ? 2 : 0);
    p.wx = mesh->d_wx;
    p.Vel = mesh->d_V;
    p.tile_variant[DST_FP64] = mesh->tile_variant[DST_FP64];
    p.tile_variant[DST_FP32] = mesh->tile_variant[DST_FP32];
    return p;
}

int dst_internal_tile_variants(const dst_mesh *mesh) { return mesh->d == 3 ? 2 : 3; }

int dst_internal_tune(dst_mesh *mesh, void *scratch, cudaStream_t s) {
    const int nv = dst_internal_tile_variants(mesh);
    mesh->tuned = true;
    if (nv <= 1 || mesh->v_general) return DST_OK;     // one shape only / the general-potential kernel
    const int64_t n = mesh->n_unknowns;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DST_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DST_ERR_CUDA;
    }
    int rc = DST_OK;
    for (int prec = 0; prec < 2 && rc == DST_OK; ++prec) {
        const size_t esz = prec == DST_FP64 ? 16 : 8;
        char *x = static_cast<char *>(scratch), *y = x + esz * n;
        if (cudaMemsetAsync(x, 0, esz * n, s) != cudaSuccess) { rc = DST_ERR_CUDA; break; }
        float best = 0.f;
        int best_v = 0;
        for (int v = 0; v < nv && rc == DST_OK; ++v) {
            mesh->tile_variant[prec] = v;
            rc = dst_internal_apply(mesh, prec, x, y, s);            // warm-up (and kernel attributes)
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && rc == DST_OK; ++r) rc = dst_internal_apply(mesh, prec, x, y, s);
            cudaEventRecord(e1, s);
            if (rc == DST_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = DST_ERR_CUDA;
            float t = 0.f;
            if (rc == DST_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = DST_ERR_CUDA;
            if (rc == DST_OK && (v == 0 || t < best)) { best = t; best_v = v; }
        }
        mesh->tile_variant[prec] = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int dst_tune_apply(dst_mesh *mesh, void *stream) {
    if (!mesh) return DST_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    if (cudaMallocAsync(&scratch, (size_t)32 * mesh->n_unknowns, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    const int rc = dst_internal_tune(mesh, scratch, s);
    cudaFreeAsync(scratch, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (rc != DST_OK) return rc;
    DST_CUDA_TRY(e);
    return DST_OK;
}

extern "C" int dst_set_apply_variant(dst_mesh *mesh, int precision, int variant) {
    if (!mesh || (precision != DST_FP64 && precision != DST_FP32) || variant < 0 ||
        variant >= dst_internal_tile_variants(mesh))
        return DST_ERR_ARG;
    mesh->tile_variant[precision] = variant;
    mesh->tuned = true;
    return DST_OK;
}

extern "C" int dst_get_apply_variant(const dst_mesh *mesh, int precision, int *variant, int *count) {
    if (!mesh || (precision != DST_FP64 && precision != DST_FP32)) return DST_ERR_ARG;
    if (variant) *variant = mesh->tile_variant[precision];
    if (count) *count = dst_internal_tile_variants(mesh);
    return DST_OK;
}

// Separable weights (m*beta + V_ex) per x element for beta = +1 and -1.  Only
// valid when V does not vary along y and z (or is zero).  Building them is the
// only step that can run out of host memory; uploading changes the mesh.
static int build_weights(const dst_mesh *mesh, double m, const std::vector<double> &V, std::vector<double> &w) {
    const int64_t nx = mesh->nel[0];
    try {
        w.resize(2 * nx);
    } catch (const std::exception &ex) {
        dst_internal_set_exception_detail("dst weights", ex.what());
        return DST_ERR_OOM;
    }
    for (int64_t e = 0; e < nx; ++e) {
        double v = V.empty() ? 0.0 : V[e];
        w[e] = m + v;
        w[nx + e] = -m + v;
    }
    return DST_OK;
}

static int upload_weights(dst_mesh *mesh, const std::vector<double> &w) {
    int dev_prev;
    DST_CUDA_TRY(cudaGetDevice(&dev_prev));
    DST_CUDA_TRY(cudaSetDevice(mesh->device));
    cudaError_t e = cudaMemcpy(mesh->d_wx, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
    cudaSetDevice(dev_prev);
    DST_CUDA_TRY(e);
    return DST_OK;
}

int dst_internal_update_weights(dst_mesh *mesh) {
    std::vector<double> w;
    const int rc = build_weights(mesh, mesh->m, mesh->V, w);
    return rc != DST_OK ? rc : upload_weights(mesh, w);
}

extern "C" int dst_create_mesh(int d, const int64_t n_el[4], const double lo[4], const double hi[4],
                               const int bc[3], dst_mesh **out) {
    if (!out || !n_el || !lo || !hi || !bc) return DST_ERR_ARG;
    *out = nullptr;
    if (d < 1 || d > 3) return DST_ERR_ARG;
    if (n_el[3] < 1 || !(hi[3] > lo[3]) || !std::isfinite(lo[3]) || !std::isfinite(hi[3])) return DST_ERR_ARG;
    for (int k = 0; k < d; ++k) {
        if (bc[k] < DST_BC_PERIODIC || bc[k] > DST_BC_DIRICHLET) return DST_ERR_ARG;
        if (n_el[k] < 1 || (bc[k] == DST_BC_DIRICHLET && n_el[k] < 2)) return DST_ERR_ARG;
        if (!(hi[k] > lo[k]) || !std::isfinite(lo[k]) || !std::isfinite(hi[k])) return DST_ERR_ARG;
    }
    int dev;
    DST_CUDA_TRY(cudaGetDevice(&dev));
    dst_mesh *m = new (std::nothrow) dst_mesh();
    if (!m) return DST_ERR_OOM;
    m->device = dev;
    m->d = d;
    m->nc = d < 3 ? 2 : 4;
    m->nt = n_el[3];
    m->lo[3] = lo[3];
    m->hi[3] = hi[3];
    m->ht = (hi[3] - lo[3]) / (double)n_el[3];
    m->n_spatial = 1;
    for (int k = 0; k < 3; ++k) {
        if (k < d) {
            m->nel[k] = n_el[k];
            m->lo[k] = lo[k];
            m->hi[k] = hi[k];
            m->bc[k] = bc[k];
            m->h[k] = (hi[k] - lo[k]) / (double)n_el[k];
            if (bc[k] == DST_BC_PERIODIC) { m->nu[k] = n_el[k]; m->u0[k] = 0; }
            else if (bc[k] == DST_BC_OPEN) { m->nu[k] = n_el[k] + 1; m->u0[k] = 0; }
            else { m->nu[k] = n_el[k] - 1; m->u0[k] = 1; }
        } else {
            m->nel[k] = 1; m->lo[k] = 0; m->hi[k] = 1; m->bc[k] = DST_BC_PERIODIC;
            m->h[k] = 1.0; m->nu[k] = 1; m->u0[k] = 0;
        }
        m->n_spatial *= m->nu[k];
    }
    m->n_unknowns = m->n_spatial * m->nt * m->nc;
    m->m = 1.0;
    m->v_general = false;
    m->d_wx = nullptr;
    m->d_V = nullptr;
    m->d_psi0 = nullptr;
    m->d_bd = nullptr;
    m->unet = nullptr;
    m->d_jac = nullptr;
    m->jac_valid = false;
    m->ws = nullptr;
    m->host_pinned = nullptr;
    m->tile_variant[0] = m->tile_variant[1] = 0;
    m->tuned = false;
    m->ws_bytes = 0;
    if (cudaMalloc(&m->d_wx, sizeof(double) * 2 * m->nel[0]) != cudaSuccess) {
        delete m;
        return DST_ERR_OOM;
    }
    int rc = dst_internal_update_weights(m);
    if (rc != DST_OK) {
        dst_destroy_mesh(m);
        return rc;
    }
    *out = m;
    return DST_OK;
}

extern "C" int dst_destroy_mesh(dst_mesh *mesh) {
    if (!mesh) return DST_OK;
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(mesh->device);
    cudaFree(mesh->d_wx);
    cudaFree(mesh->d_V);
    cudaFree(mesh->d_psi0);
    cudaFree(mesh->d_bd);
    cudaFree(mesh->d_jac);
    cudaFree(mesh->ws);
    if (mesh->host_pinned) cudaFreeHost(mesh->host_pinned);
    cudaSetDevice(dev_prev);
    delete mesh;
    return DST_OK;
}

extern "C" int dst_mesh_sizes(const dst_mesh *mesh, int64_t *n_spatial_nodes, int64_t *n_unknowns, int *ncomp) {
    if (!mesh) return DST_ERR_ARG;
    if (n_spatial_nodes) *n_spatial_nodes = mesh->n_spatial;
    if (n_unknowns) *n_unknowns = mesh->n_unknowns;
    if (ncomp) *ncomp = mesh->nc;
    return DST_OK;
}

extern "C" int dst_set_mass(dst_mesh *mesh, double m) {
    if (!mesh || !std::isfinite(m)) return DST_ERR_ARG;
    std::vector<double> w;
    int rc = build_weights(mesh, m, mesh->V, w);
    if (rc == DST_OK) rc = upload_weights(mesh, w);
    if (rc == DST_OK) {
        mesh->m = m;
        mesh->jac_valid = false;      // the Jacobi blocks depend on the operator
    }
    return rc;
}

// The mesh changes only once every step that can fail for want of memory has
// succeeded, so that DST_ERR_OOM leaves the previous potential in force and a
// general potential never goes without its device copy.
static int set_potential(dst_mesh *mesh, const double *V_elem) {
    const int64_t nx = mesh->nel[0], nyz = mesh->nel[1] * mesh->nel[2];
    const int64_t ne = V_elem ? nx * nyz : 0;
    for (int64_t i = 0; i < ne; ++i)
        if (!std::isfinite(V_elem[i])) return DST_ERR_ARG;
    std::vector<double> V(V_elem, V_elem + ne), w;
    bool general = false;
    for (int64_t j = 1; j < nyz && ne && !general; ++j)
        for (int64_t e = 0; e < nx; ++e)
            if (V_elem[j * nx + e] != V_elem[e]) { general = true; break; }
    int rc = build_weights(mesh, mesh->m, V, w);
    if (rc != DST_OK) return rc;
    if (general) {
        int dev_prev;
        DST_CUDA_TRY(cudaGetDevice(&dev_prev));
        DST_CUDA_TRY(cudaSetDevice(mesh->device));
        if (!mesh->d_V && cudaMalloc(&mesh->d_V, sizeof(double) * ne) != cudaSuccess) {
            cudaGetLastError();
            mesh->d_V = nullptr;
            cudaSetDevice(dev_prev);
            return DST_ERR_OOM;
        }
        cudaError_t e = cudaMemcpy(mesh->d_V, V_elem, sizeof(double) * ne, cudaMemcpyHostToDevice);
        cudaSetDevice(dev_prev);
        DST_CUDA_TRY(e);
    }
    if ((rc = upload_weights(mesh, w)) != DST_OK) return rc;
    mesh->V.swap(V);
    mesh->v_general = general;
    mesh->jac_valid = false;
    return DST_OK;
}

extern "C" int dst_set_potential(dst_mesh *mesh, const double *V_elem) {
    if (!mesh) return DST_ERR_ARG;
    return dst_internal_guard("dst_set_potential", [&] { return set_potential(mesh, V_elem); });
}

static int set_initial_data(dst_mesh *mesh, const double *psi0) {
    const int64_t n = mesh->n_spatial * mesh->nc * 2;
    mesh->psi0.assign(psi0, psi0 + n);
    int dev_prev;
    DST_CUDA_TRY(cudaGetDevice(&dev_prev));
    DST_CUDA_TRY(cudaSetDevice(mesh->device));
    if (!mesh->d_psi0 && cudaMalloc(&mesh->d_psi0, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        mesh->d_psi0 = nullptr;
        cudaSetDevice(dev_prev);
        return DST_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(mesh->d_psi0, psi0, sizeof(double) * n, cudaMemcpyHostToDevice);
    cudaSetDevice(dev_prev);
    DST_CUDA_TRY(e);
    return DST_OK;
}

extern "C" int dst_set_initial_data(dst_mesh *mesh, const double *psi0) {
    if (!mesh || !psi0) return DST_ERR_ARG;
    return dst_internal_guard("dst_set_initial_data", [&] { return set_initial_data(mesh, psi0); });
}

double dst_internal_apply_flops(const dst_mesh *mesh) {
    static const double base[4] = {0.0, 26.0, 44.0, 68.0}, pot[4] = {0.0, 10.0, 16.0, 22.0};
    const double per = base[mesh->d] + (mesh->V.empty() ? 0.0 : pot[mesh->d]);
    return per * (double)mesh->n_unknowns;
}

int dst_internal_apply(const dst_mesh *mesh, int precision, const void *x, void *y, cudaStream_t s) {
    OpParams p = dst_internal_params(mesh);
    switch (mesh->d) {
        case 1: return dst_launch_apply_d1(p, precision, x, y, s);
        case 2: return dst_launch_apply_d2(p, precision, x, y, s);
        default: return dst_launch_apply_d3(p, precision, x, y, s);
    }
}

int dst_internal_rhs(const dst_mesh *mesh, double2 *b, cudaStream_t s) {
    OpParams p = dst_internal_params(mesh);
    int rc;
    switch (mesh->d) {
        case 1: rc = dst_launch_rhs_d1(p, mesh->d_psi0, b, s); break;
        case 2: rc = dst_launch_rhs_d2(p, mesh->d_psi0, b, s); break;
        default: rc = dst_launch_rhs_d3(p, mesh->d_psi0, b, s); break;
    }
    return rc != DST_OK ? rc : dst_internal_rhs_walls(mesh, b, s);
}

extern "C" int dst_apply_operator(const dst_mesh *mesh, int precision, const void *x, void *y, void *stream) {
    if (!mesh || !x || !y || (precision != DST_FP64 && precision != DST_FP32)) return DST_ERR_ARG;
    if (x == y) return DST_ERR_ARG;
    if (((uintptr_t)x | (uintptr_t)y) & 15) {
        dst_internal_set_error_detail("dst_apply_operator: x and y must be 16-byte aligned");
        return DST_ERR_ARG;
    }
    return dst_internal_apply(mesh, precision, x, y, (cudaStream_t)stream);
}

extern "C" int dst_build_rhs(const dst_mesh *mesh, void *b, void *stream) {
    if (!mesh || !b) return DST_ERR_ARG;
    if (!mesh->d_psi0) return DST_ERR_STATE;
    return dst_internal_rhs(mesh, (double2 *)b, (cudaStream_t)stream);
}
