// Internal declarations of the diracst library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <vector>

#include "../../include/diracst.h"

#define DST_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            dst_internal_set_cuda_error(e_, #expr, __FILE__, __LINE__); \
            return DST_ERR_CUDA;                             \
        }                                                    \
    } while (0)

void dst_internal_set_cuda_error(cudaError_t e, const char *expr, const char *file, int line);
void dst_internal_set_error_detail(const char *msg);
void dst_internal_set_exception_detail(const char *call, const char *what);

// Runs the body of a C ABI entry point that allocates host memory or starts
// host threads, so that no C++ exception crosses the C ABI: the only ones these
// bodies can raise are a failed host allocation or thread start, returned as
// DST_ERR_OOM with the exception's text as the error detail.
template <class F>
int dst_internal_guard(const char *call, F &&body) noexcept {
    try {
        return body();
    } catch (const std::exception &e) {
        dst_internal_set_exception_detail(call, e.what());
    } catch (...) {
        dst_internal_set_exception_detail(call, "unknown C++ exception");
    }
    return DST_ERR_OOM;
}

// Geometry of one spatial axis, as the kernels see it.
struct AxisDesc {
    int64_t n;      // unknown nodes along the axis
    int64_t nel;    // elements along the axis
    int bc;         // DST_BC_*
    int u0;         // geometric index of unknown node 0 (1 for Dirichlet, else 0)
    double h;       // element size
};

// Everything an operator-apply kernel needs, passed by value.
struct OpParams {
    AxisDesc ax[3];          // x, y, z (unused axes: n = nel = 1, periodic)
    int64_t nt;              // unknown time layers N_t
    double ht;               // time element size
    double m;                // mass
    int vmode;               // 0: x-only weights, 1: general per-element V, 2: no potential
    const double *wx;        // separable: [2*nel_x]: (m + V_ex) then (-m + V_ex)
    const double *Vel;       // general: V per spatial element (x fastest)
    int tile_variant[2];     // apply tile shape per precision (index DST_FP64 / DST_FP32)
};

struct dst_unet;

struct dst_mesh {
    int device;
    int d, nc;
    int64_t nel[3], nt;
    double lo[4], hi[4];
    int bc[3];
    double h[3], ht;
    int64_t nu[3];
    int u0[3];
    int64_t n_spatial, n_unknowns;
    double m;
    std::vector<double> V;        // host copy, empty = zero potential
    bool v_general;               // true if V varies along y or z
    double *d_wx;                 // [2*nel_x] separable weights
    double *d_V;                  // general potential (or null)
    std::vector<double> psi0;     // host copy of the initial layer
    double2 *d_psi0;              // device copy (null until set)
    double2 *d_bd;                // Dirichlet wall values, layers 0..N_t on the open-axis node grid
                                  // (zero off the walls); null = homogeneous walls
    int tile_variant[2];          // apply tile shape per precision, set by the autotuner
    bool tuned;                   // the autotuner has run on this mesh
    // GMRES workspace (allocated lazily by dst_solve)
    void *ws;
    size_t ws_bytes;
    double *host_pinned;          // page-locked host copy of the per-step records (lazily, by dst_solve)
    dst_unet *unet;               // learned correction of the sweep preconditioner (not owned), or null
    void *d_jac;                  // inverse node blocks of the block Jacobi preconditioner (float2
                                  // [node][NC][NC]), built on first use
    bool jac_valid;               // d_jac matches the current mass and potential
};

// Node-block Jacobi preconditioner (jacobi.cu): build the inverse blocks of the
// current operator (once; synchronises s), and z = blockdiag(A_nn)^-1 v in FP32.
int dst_internal_jacobi_setup(dst_mesh *mesh, cudaStream_t s);
int dst_internal_jacobi_apply(const dst_mesh *mesh, const float2 *v, float2 *z, cudaStream_t s);

// The learned correction (unet.cu): z += alpha U(rho / ||rho||) with alpha the
// complex least-squares scale minimising ||rho - alpha A U|| (tmp: a free FP32
// vector for A U; *launches: kernels enqueued); and whether a network was
// built for this mesh's grid on its device.
int dst_internal_unet_correct(dst_unet *u, const dst_mesh *mesh, const float2 *rho, float2 *z, float2 *tmp,
                              cudaStream_t s, int *launches);
bool dst_internal_unet_fits(const dst_unet *u, const dst_mesh *mesh);

// Testing hooks (dst_testing_set): the bulk-copy wait limit in force (the
// standard one unless a test set another), and whether the next workspace
// allocation is to fail as if the device were out of memory.
unsigned dst_internal_wait_limit(unsigned standard);
bool dst_internal_injected_alloc_failure();

OpParams dst_internal_params(const dst_mesh *mesh);
int dst_internal_update_weights(dst_mesh *mesh);

// Kernel launchers, one translation unit per spatial dimension (apply_d{1,2,3}.cu).
int dst_launch_apply_d1(const OpParams &p, int precision, const void *x, void *y, cudaStream_t s);
int dst_launch_apply_d2(const OpParams &p, int precision, const void *x, void *y, cudaStream_t s);
int dst_launch_apply_d3(const OpParams &p, int precision, const void *x, void *y, cudaStream_t s);
int dst_launch_rhs_d1(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s);
int dst_launch_rhs_d2(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s);
int dst_launch_rhs_d3(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s);

// Algorithmic floating-point operations of one operator apply: per complex
// unknown, the sum-factorised evaluation (real flops, an FMA counting two):
// x stencils M, C (8); in 2+1 the y pass on them (14), in 3+1 y (14) and z (20);
// a potential's weighted mass field (10, +6 per further axis); the spin
// combination (4 + 4 d) and the two time stencils (10).  Per unknown: 26 / 44 /
// 68 in 1+1 / 2+1 / 3+1, plus 10 / 16 / 22 with a potential.
double dst_internal_apply_flops(const dst_mesh *mesh);

// Dispatch on the mesh dimension.
int dst_internal_apply(const dst_mesh *mesh, int precision, const void *x, void *y, cudaStream_t s);
int dst_internal_rhs(const dst_mesh *mesh, double2 *b, cudaStream_t s);
// b += -D_w[unknowns, wall nodes] Psi_wall when the mesh carries wall values (boundary.cu)
int dst_internal_rhs_walls(const dst_mesh *mesh, double2 *b, cudaStream_t s);
// Time every apply tile variant of both precisions on scratch (at least
// 32 * n_unknowns bytes of device memory, contents overwritten) and keep the
// fastest in mesh->tile_variant; synchronises s.
int dst_internal_tune(dst_mesh *mesh, void *scratch, cudaStream_t s);
int dst_internal_tile_variants(const dst_mesh *mesh);
