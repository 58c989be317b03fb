// Prescribed values on Dirichlet walls (Sec. 2.1, Eq. 2: Psi = Psi_0 on the
// boundary).  The known/unknown split of Eq. 11 moves every known spinor to the
// right-hand side: b = -D_w21 Psi_known.  With nonzero wall values the known
// spinors are the t = 0 layer and the end nodes of Dirichlet axes on every
// time layer, so b gains -D_w[unknowns, wall nodes] Psi_wall.
//
// The rows of the unknowns of a Dirichlet mesh are the interior rows of the
// same mesh with those axes open (natural boundary, end nodes unknown): the
// element sum that forms a row does not depend on how the end nodes are
// treated.  So the wall term is evaluated with the existing open-axis apply:
// place the wall values on the open mesh's nodes (zero elsewhere), apply the
// open operator to layers 1..N_t, take the open right-hand side of layer 0's
// wall values, and add (open RHS - open apply) at the interior nodes to b.
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

namespace {

// b[unknown node] += y1[open node] - y2[open node] over all unknown layers.
__global__ void add_wall_term_kernel(int64_t nx, int64_t ny, int64_t nz, int64_t nt, int nc, int sx, int sy, int sz,
                                     int64_t ox, int64_t oy, int64_t oz, const double2 *__restrict__ y1,
                                     const double2 *__restrict__ y2, double2 *__restrict__ b) {
    const int64_t total = nx * ny * nz * nt * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i % nc;
        int64_t r = i / nc;
        const int64_t ix = r % nx; r /= nx;
        const int64_t iy = r % ny; r /= ny;
        const int64_t iz = r % nz;
        const int64_t it = r / nz;
        const int64_t j = ((((it * oz) + iz + sz) * oy + iy + sy) * ox + ix + sx) * nc + c;
        const double2 a = y1[j], q = y2[j];
        double2 v = b[i];
        v.x += a.x - q.x;
        v.y += a.y - q.y;
        b[i] = v;
    }
}

}  // namespace

// Open-axis twin of a mesh's operator parameters: every Dirichlet axis keeps its
// elements and gets all its n_el + 1 nodes as (open) unknowns.
static OpParams open_params(const dst_mesh *mesh) {
    OpParams p = dst_internal_params(mesh);
    for (int k = 0; k < mesh->d; ++k) {
        if (mesh->bc[k] != DST_BC_DIRICHLET) continue;
        p.ax[k].bc = DST_BC_OPEN;
        p.ax[k].n = mesh->nel[k] + 1;
        p.ax[k].u0 = 0;
    }
    return p;
}

static int64_t open_spatial_nodes(const dst_mesh *mesh) {
    int64_t n = 1;
    for (int k = 0; k < 3; ++k) n *= (k < mesh->d && mesh->bc[k] == DST_BC_DIRICHLET) ? mesh->nel[k] + 1 : mesh->nu[k];
    return n;
}

int dst_internal_rhs_walls(const dst_mesh *mesh, double2 *b, cudaStream_t s) {
    if (!mesh->d_bd) return DST_OK;
    const OpParams po = open_params(mesh);
    const int64_t per = open_spatial_nodes(mesh) * mesh->nc;        // entries of one open layer
    const int64_t nopen = per * mesh->nt;
    double2 *y1 = nullptr, *y2 = nullptr;
    if (cudaMallocAsync(&y1, sizeof(double2) * nopen, s) != cudaSuccess ||
        cudaMallocAsync(&y2, sizeof(double2) * nopen, s) != cudaSuccess) {
        cudaGetLastError();
        if (y1) cudaFreeAsync(y1, s);
        dst_internal_set_error_detail("dst_build_rhs: no device memory for the wall term");
        return DST_ERR_OOM;
    }
    int rc;
    switch (mesh->d) {
        case 1: rc = dst_launch_rhs_d1(po, mesh->d_bd, y1, s); break;
        case 2: rc = dst_launch_rhs_d2(po, mesh->d_bd, y1, s); break;
        default: rc = dst_launch_rhs_d3(po, mesh->d_bd, y1, s); break;
    }
    if (rc == DST_OK) {
        const double2 *x = mesh->d_bd + per;                         // wall values of layers 1..N_t
        switch (mesh->d) {
            case 1: rc = dst_launch_apply_d1(po, DST_FP64, x, y2, s); break;
            case 2: rc = dst_launch_apply_d2(po, DST_FP64, x, y2, s); break;
            default: rc = dst_launch_apply_d3(po, DST_FP64, x, y2, s); break;
        }
    }
    if (rc == DST_OK) {
        auto shift = [&](int k) { return (k < mesh->d && mesh->bc[k] == DST_BC_DIRICHLET) ? 1 : 0; };
        add_wall_term_kernel<<<1024, 256, 0, s>>>(mesh->nu[0], mesh->nu[1], mesh->nu[2], mesh->nt, mesh->nc, shift(0),
                                                  shift(1), shift(2), po.ax[0].n, po.ax[1].n, po.ax[2].n, y1, y2, b);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            dst_internal_set_cuda_error(e, "add_wall_term_kernel", __FILE__, __LINE__);
            rc = DST_ERR_CUDA;
        }
    }
    cudaFreeAsync(y1, s);
    cudaFreeAsync(y2, s);
    return rc;
}

// Keep the values on Dirichlet end nodes of every layer, zero elsewhere, and
// upload them; the mesh changes only after every step that can fail.
static int set_boundary_data(dst_mesh *mesh, const double *psi_bd) {
    bool any = false;
    for (int k = 0; k < mesh->d; ++k) any = any || mesh->bc[k] == DST_BC_DIRICHLET;
    if (!any) {
        dst_internal_set_error_detail("dst_set_boundary_data: the mesh has no Dirichlet axis");
        return DST_ERR_ARG;
    }
    int dev_prev;
    DST_CUDA_TRY(cudaGetDevice(&dev_prev));
    if (!psi_bd) {
        DST_CUDA_TRY(cudaSetDevice(mesh->device));
        cudaFree(mesh->d_bd);
        mesh->d_bd = nullptr;
        cudaSetDevice(dev_prev);
        return DST_OK;
    }
    int64_t g[3];
    for (int k = 0; k < 3; ++k) g[k] = (k < mesh->d && mesh->bc[k] == DST_BC_DIRICHLET) ? mesh->nel[k] + 1 : mesh->nu[k];
    const int nc = mesh->nc;
    const int64_t per = g[0] * g[1] * g[2] * nc;
    const int64_t total = per * (mesh->nt + 1);
    std::vector<double> h((size_t)(2 * total), 0.0);
    for (int64_t t = 0; t <= mesh->nt; ++t)
        for (int64_t z = 0; z < g[2]; ++z)
            for (int64_t y = 0; y < g[1]; ++y)
                for (int64_t x = 0; x < g[0]; ++x) {
                    const int64_t c3[3] = {x, y, z};
                    bool wall = false;
                    for (int k = 0; k < mesh->d; ++k)
                        wall = wall || (mesh->bc[k] == DST_BC_DIRICHLET && (c3[k] == 0 || c3[k] == g[k] - 1));
                    if (!wall) continue;
                    const int64_t base = 2 * ((((t * g[2] + z) * g[1] + y) * g[0] + x) * nc);
                    for (int q = 0; q < 2 * nc; ++q) {
                        const double v = psi_bd[base + q];
                        if (!std::isfinite(v)) {
                            dst_internal_set_error_detail("dst_set_boundary_data: non-finite wall value");
                            return DST_ERR_ARG;
                        }
                        h[(size_t)(base + q)] = v;
                    }
                }
    DST_CUDA_TRY(cudaSetDevice(mesh->device));
    double2 *d = nullptr;
    if (cudaMalloc(&d, sizeof(double2) * total) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(dev_prev);
        return DST_ERR_OOM;
    }
    const cudaError_t e = cudaMemcpy(d, h.data(), sizeof(double2) * total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        cudaSetDevice(dev_prev);
        DST_CUDA_TRY(e);
    }
    cudaFree(mesh->d_bd);
    mesh->d_bd = d;
    cudaSetDevice(dev_prev);
    return DST_OK;
}

extern "C" int dst_set_boundary_data(dst_mesh *mesh, const double *psi_bd) {
    if (!mesh) return DST_ERR_ARG;
    return dst_internal_guard("dst_set_boundary_data", [&] { return set_boundary_data(mesh, psi_bd); });
}
