// Node-block Jacobi preconditioner: z = blockdiag(A_nn)^-1 v, with A_nn the
// NC x NC block of D_w22 (Eq. 11) that couples the spinor components of unknown
// node n with themselves.  The paper names no preconditioner (its conclusion,
// Sec. 5, asks for one); this is the classical comparator for the sweep and
// the learned correction.
//
// The blocks are read off the operator itself by probing.  The sum-factorised
// stencil couples a node only with nodes at most one step away along every
// axis (t included), so in a colouring where any two nodes of one colour are
// two or more steps apart along some axis - i mod 3 per axis; on a periodic
// axis whose length is not a multiple of 3 the last n mod 3 nodes get colours
// of their own - applying A to the indicator of one colour and one component c'
// returns, at every node of that colour, column c' of its block.  That is
// (colours) x NC FP32 applies once per mesh (81 x 4 for the 3+1 Klein mesh),
// every boundary and potential handled by the apply itself; the blocks are
// inverted in FP64 (Gauss-Jordan with partial pivoting) and stored in FP32.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace {

struct JacGeom {
    int64_t n[4];      // nodes along x, y, z, t (unknown layers)
    int r[4];          // periodic remainder n mod 3 (0 otherwise): colours 3 .. 2 + r
    int ncol[4];       // colours per axis
    int64_t ncolor;    // product
};

__device__ __forceinline__ int axis_colour(int64_t i, int64_t n, int r) {
    return i < n - r ? (int)(i % 3) : 3 + (int)(i - (n - r));
}

// colour of unknown node `node` (layout [t][z][y][x])
__device__ __forceinline__ int64_t node_colour(const JacGeom &g, int64_t node) {
    const int64_t x = node % g.n[0];
    int64_t q = node / g.n[0];
    const int64_t y = q % g.n[1];
    q /= g.n[1];
    const int64_t z = q % g.n[2];
    const int64_t t = q / g.n[2];
    int64_t c = axis_colour(t, g.n[3], g.r[3]);
    c = c * g.ncol[2] + axis_colour(z, g.n[2], g.r[2]);
    c = c * g.ncol[1] + axis_colour(y, g.n[1], g.r[1]);
    return c * g.ncol[0] + axis_colour(x, g.n[0], g.r[0]);
}

__global__ void probe_kernel(int64_t nodes, int nc, JacGeom g, int64_t colour, int comp, float2 *__restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nodes * nc;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t node = i / nc;
        const bool on = (int)(i % nc) == comp && node_colour(g, node) == colour;
        x[i] = make_float2(on ? 1.f : 0.f, 0.f);
    }
}

// column `comp` of the blocks of the nodes of one colour: blocks[node][row][comp] = y[node][row]
__global__ void extract_kernel(int64_t nodes, int nc, JacGeom g, int64_t colour, int comp,
                               const float2 *__restrict__ y, double2 *__restrict__ blocks) {
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nodes;
         node += (int64_t)gridDim.x * blockDim.x) {
        if (node_colour(g, node) != colour) continue;
        for (int r = 0; r < nc; ++r) {
            const float2 a = y[node * nc + r];
            blocks[(node * nc + r) * nc + comp] = make_double2(a.x, a.y);
        }
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cinv(double2 a) {
    const double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}

// inverse of every NC x NC block (NC <= 4), FP64 Gauss-Jordan with partial pivoting,
// stored in FP32; a block whose pivot vanishes (|pivot| <= 1e-13 of its largest entry)
// is replaced by the identity (no preconditioning at that node)
template <int NC>
__global__ void invert_kernel(int64_t nodes, const double2 *__restrict__ blocks, float2 *__restrict__ binv) {
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nodes;
         node += (int64_t)gridDim.x * blockDim.x) {
        double2 a[NC][NC], b[NC][NC];
        double amax = 0.0;
#pragma unroll
        for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                a[i][j] = blocks[(node * NC + i) * NC + j];
                b[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
                amax = fmax(amax, hypot(a[i][j].x, a[i][j].y));
            }
        bool ok = amax > 0.0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            int p = k;
            double pm = hypot(a[k][k].x, a[k][k].y);
#pragma unroll
            for (int i = k + 1; i < NC; ++i) {
                const double v = hypot(a[i][k].x, a[i][k].y);
                if (v > pm) { pm = v; p = i; }
            }
            if (!(pm > 1e-13 * amax)) ok = false;
            if (!ok) continue;
#pragma unroll
            for (int j = 0; j < NC; ++j) {         // swap rows k and p (unrolled: registers)
                if (p == k) break;
#pragma unroll
                for (int i = k + 1; i < NC; ++i) {
                    if (i != p) continue;
                    const double2 ta = a[k][j], tb = b[k][j];
                    a[k][j] = a[i][j]; b[k][j] = b[i][j];
                    a[i][j] = ta; b[i][j] = tb;
                }
            }
            const double2 inv = cinv(a[k][k]);
#pragma unroll
            for (int j = 0; j < NC; ++j) { a[k][j] = cmul(a[k][j], inv); b[k][j] = cmul(b[k][j], inv); }
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                if (i == k) continue;
                const double2 f = a[i][k];
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    const double2 fa = cmul(f, a[k][j]), fb = cmul(f, b[k][j]);
                    a[i][j].x -= fa.x; a[i][j].y -= fa.y;
                    b[i][j].x -= fb.x; b[i][j].y -= fb.y;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const double2 v = ok ? b[i][j] : make_double2(i == j ? 1.0 : 0.0, 0.0);
                binv[(node * NC + i) * NC + j] = make_float2((float)v.x, (float)v.y);
            }
    }
}

// z_n = Binv_n v_n
template <int NC>
__global__ void __launch_bounds__(256) jacobi_apply_kernel(int64_t nodes, const float2 *__restrict__ binv,
                                                           const float2 *__restrict__ v, float2 *__restrict__ z) {
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < nodes;
         node += (int64_t)gridDim.x * blockDim.x) {
        float2 x[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) x[j] = v[node * NC + j];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const float2 m = binv[(node * NC + i) * NC + j];
                acc.x = fmaf(m.x, x[j].x, fmaf(-m.y, x[j].y, acc.x));
                acc.y = fmaf(m.x, x[j].y, fmaf(m.y, x[j].x, acc.y));
            }
            z[node * NC + i] = acc;
        }
    }
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 16 * 152) b = 16 * 152;
    return (unsigned)(b < 1 ? 1 : b);
}

JacGeom geometry(const dst_mesh *mesh) {
    JacGeom g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < mesh->d ? mesh->nu[a] : 1;
        const bool per = a < mesh->d && mesh->bc[a] == DST_BC_PERIODIC;
        g.r[a] = per && g.n[a] > 3 ? (int)(g.n[a] % 3) : 0;
    }
    g.n[3] = mesh->nt;
    g.r[3] = 0;
    g.ncolor = 1;
    for (int a = 0; a < 4; ++a) {
        g.ncol[a] = (g.n[a] < 3 ? (int)g.n[a] : 3) + g.r[a];
        g.ncolor *= g.ncol[a];
    }
    return g;
}

}  // namespace

int dst_internal_jacobi_setup(dst_mesh *mesh, cudaStream_t s) {
    if (mesh->d_jac && mesh->jac_valid) return DST_OK;
    const int nc = mesh->nc;
    const int64_t nodes = mesh->nt * mesh->n_spatial, n = mesh->n_unknowns;
    if (!mesh->d_jac && cudaMalloc(&mesh->d_jac, sizeof(float2) * (size_t)nodes * nc * nc) != cudaSuccess) {
        cudaGetLastError();
        mesh->d_jac = nullptr;
        return DST_ERR_OOM;
    }
    // scratch: the probe and its image (FP32 vectors), the FP64 blocks
    char *scr = nullptr;
    const size_t vb = ((size_t)n * sizeof(float2) + 255) & ~(size_t)255;
    const size_t bb = ((size_t)nodes * nc * nc * sizeof(double2) + 255) & ~(size_t)255;
    if (cudaMallocAsync((void **)&scr, 2 * vb + bb, s) != cudaSuccess) {
        cudaGetLastError();
        return DST_ERR_OOM;
    }
    float2 *x = reinterpret_cast<float2 *>(scr), *y = reinterpret_cast<float2 *>(scr + vb);
    double2 *blocks = reinterpret_cast<double2 *>(scr + 2 * vb);
    const JacGeom g = geometry(mesh);
    int rc = DST_OK;
    for (int64_t c = 0; c < g.ncolor && rc == DST_OK; ++c)
        for (int comp = 0; comp < nc && rc == DST_OK; ++comp) {
            probe_kernel<<<grid_for(n), 256, 0, s>>>(nodes, nc, g, c, comp, x);
            rc = dst_internal_apply(mesh, DST_FP32, x, y, s);
            if (rc == DST_OK) extract_kernel<<<grid_for(nodes), 256, 0, s>>>(nodes, nc, g, c, comp, y, blocks);
        }
    if (rc == DST_OK) {
        float2 *binv = reinterpret_cast<float2 *>(mesh->d_jac);
        if (nc == 2) invert_kernel<2><<<grid_for(nodes), 128, 0, s>>>(nodes, blocks, binv);
        else invert_kernel<4><<<grid_for(nodes), 128, 0, s>>>(nodes, blocks, binv);
    }
    if (rc == DST_OK && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess))
        rc = DST_ERR_CUDA;
    cudaFreeAsync(scr, s);
    if (rc != DST_OK) return rc;
    mesh->jac_valid = true;
    return DST_OK;
}

int dst_internal_jacobi_apply(const dst_mesh *mesh, const float2 *v, float2 *z, cudaStream_t s) {
    if (!mesh->d_jac || !mesh->jac_valid) return DST_ERR_STATE;
    const int64_t nodes = mesh->nt * mesh->n_spatial;
    const float2 *binv = reinterpret_cast<const float2 *>(mesh->d_jac);
    if (mesh->nc == 2) jacobi_apply_kernel<2><<<grid_for(nodes), 256, 0, s>>>(nodes, binv, v, z);
    else jacobi_apply_kernel<4><<<grid_for(nodes), 256, 0, s>>>(nodes, binv, v, z);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}
