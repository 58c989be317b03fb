// Observables of a solution per time layer (Sec. 4.2 Eq. 20, Sec. 4.3 Eq. 25):
// charge, charge right of a point, first moments, by trapezoidal sums.
// One CTA per time layer; each thread sums a fixed strided subset of the
// layer's nodes, then a fixed-order block reduction (deterministic).
#include "internal.h"

namespace {

constexpr int OBS_THREADS = 512;

struct AxisGeo {
    int64_t n;       // unknown nodes
    int u0;          // geometric index of unknown node 0
    int open;        // 1: halve the end nodes
    double lo, h;
};

__device__ __forceinline__ double axis_weight(const AxisGeo &a, int64_t i) {
    if (a.open && (i == 0 || i == a.n - 1)) return 0.5 * a.h;
    return a.h;
}

__global__ void __launch_bounds__(OBS_THREADS)
observables_kernel(AxisGeo ax, AxisGeo ay, AxisGeo az, int d, int nc, const double2 *__restrict__ psi, double x0,
                   double *__restrict__ out) {
    __shared__ double red[OBS_THREADS / 32][5];
    const int64_t layer = blockIdx.x;
    const int64_t ns = ax.n * ay.n * az.n;
    const double2 *p = psi + layer * ns * nc;
    double q = 0.0, qr = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int64_t s = threadIdx.x; s < ns; s += OBS_THREADS) {
        const int64_t ix = s % ax.n, iy = (s / ax.n) % ay.n, iz = s / (ax.n * ay.n);
        double rho = 0.0;
        for (int c = 0; c < nc; ++c) {
            const double2 v = p[s * nc + c];
            rho = fma(v.x, v.x, fma(v.y, v.y, rho));
        }
        double w = axis_weight(ax, ix);
        if (d >= 2) w *= axis_weight(ay, iy);
        if (d >= 3) w *= axis_weight(az, iz);
        const double x = ax.lo + ax.h * (double)(ax.u0 + ix);
        const double wr = w * rho;
        q += wr;
        qr += x > x0 + 1e-12 ? wr : (x < x0 - 1e-12 ? 0.0 : 0.5 * wr);
        mx = fma(x, wr, mx);
        if (d >= 2) my = fma(ay.lo + ay.h * (double)(ay.u0 + iy), wr, my);
        if (d >= 3) mz = fma(az.lo + az.h * (double)(az.u0 + iz), wr, mz);
    }
    double vals[5] = {q, qr, mx, my, mz};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double v = vals[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < OBS_THREADS / 32; ++w) t += red[w][threadIdx.x];
        out[layer * 5 + threadIdx.x] = t;
    }
}

AxisGeo geo(const dst_mesh *m, int k) {
    AxisGeo a;
    a.n = m->nu[k];
    a.u0 = m->u0[k];
    a.open = (k < m->d && m->bc[k] == DST_BC_OPEN) ? 1 : 0;
    a.lo = m->lo[k];
    a.h = m->h[k];
    return a;
}

}  // namespace

extern "C" int dst_observables(const dst_mesh *mesh, const void *psi, double x0, void *out, void *stream) {
    if (!mesh || !psi || !out || mesh->nt > 0x7fffffffLL) return DST_ERR_ARG;
    observables_kernel<<<(unsigned)mesh->nt, OBS_THREADS, 0, (cudaStream_t)stream>>>(
        geo(mesh, 0), geo(mesh, 1), geo(mesh, 2), mesh->d, mesh->nc, (const double2 *)psi, x0, (double *)out);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}
