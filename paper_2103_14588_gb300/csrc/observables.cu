// Observables of a solution per time layer (Sec. 4.2 Eq. 20, Sec. 4.3 Eq. 25):
// charge, charge right of a point, first moments, by trapezoidal sums.
// One CTA per time layer; each thread sums a fixed strided subset of the
// layer's nodes, then a fixed-order block reduction (deterministic).
// The energy per layer (the other reading of Sec. 4.1's E(t)) applies the free
// Dirac Hamiltonian spectrally on periodic meshes: FP64 FFT of every layer, then
// sum over frequencies of psi^ dagger H(p) psi^ (Parseval).
#include "fft.cuh"
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

// Energy of each layer from its FFT: (prod h) / nf * sum_f Re(psi^_f^dagger H(p_f) psi^_f),
// H(p) = sum_k alpha_k p_k + beta m, p_k = 2 pi q_k / (n_k h_k) with q_k the signed
// frequency of index f_k (f_k < (n_k + 1) / 2 positive, else f_k - n_k).  Entry layout
// of psi^: [t][f][c], f = fy nx + fx (1+1, 2+1) or (fy nx + fx) nz + fz (3+1, two passes).
struct EGeo {
    int d, nc;
    int n[3];          // nodes per axis (x, y, z)
    double h[3];
    double m;
    int64_t nf;        // frequencies per layer
};

__device__ __forceinline__ double signed_freq(int f, int n) { return (double)(f < (n + 1) / 2 ? f : f - n); }

__global__ void __launch_bounds__(OBS_THREADS)
energy_kernel(EGeo g, const double2 *__restrict__ ph, double *__restrict__ out) {
    __shared__ double red[OBS_THREADS / 32];
    const int64_t layer = blockIdx.x;
    const double2 *p = ph + layer * g.nf * g.nc;
    const double PI2 = 6.283185307179586476925;
    double acc = 0.0;
    for (int64_t f = threadIdx.x; f < g.nf; f += OBS_THREADS) {
        // d = 1, 2: f = fy * nx + fx;  d = 3: f = (fy * nx + fx) * nz + fz (two FFT passes)
        int fx, fy = 0, fz = 0;
        if (g.d == 3) {
            fz = (int)(f % g.n[2]);
            const int64_t fyx = f / g.n[2];
            fx = (int)(fyx % g.n[0]);
            fy = (int)(fyx / g.n[0]);
        } else {
            fx = (int)(f % g.n[0]);
            fy = (int)(f / g.n[0]);
        }
        const double pk[3] = {PI2 * signed_freq(fx, g.n[0]) / (g.n[0] * g.h[0]),
                              g.d >= 2 ? PI2 * signed_freq(fy, g.n[1]) / (g.n[1] * g.h[1]) : 0.0,
                              g.d >= 3 ? PI2 * signed_freq(fz, g.n[2]) / (g.n[2] * g.h[2]) : 0.0};
        double2 v[4];
        for (int c = 0; c < g.nc; ++c) v[c] = p[f * g.nc + c];
        for (int c = 0; c < g.nc; ++c) {
            // (H v)_c = beta_c m v_c + sum_k p_k phi_k(c) v_{pi_k(c)}
            const double bc = g.nc == 2 ? (c == 0 ? 1.0 : -1.0) : (c < 2 ? 1.0 : -1.0);
            double hx = bc * g.m * v[c].x, hy = bc * g.m * v[c].y;
            for (int k = 0; k < g.d; ++k) {
                const int q = g.nc == 2 ? 1 - c : (k == 2 ? (c + 2) & 3 : 3 - c);
                const double2 u = v[q];
                double ux, uy;                                   // phi_k(c) u
                if (k == 0) { ux = u.x; uy = u.y; }
                else if (k == 1) {                               // sigma_y rows: -i, +i
                    if (c & 1) { ux = -u.y; uy = u.x; } else { ux = u.y; uy = -u.x; }
                } else {                                         // sigma_z in the off-diagonal blocks
                    if (c & 1) { ux = -u.x; uy = -u.y; } else { ux = u.x; uy = u.y; }
                }
                hx = fma(pk[k], ux, hx);
                hy = fma(pk[k], uy, hy);
            }
            acc += v[c].x * hx + v[c].y * hy;                    // Re(conj(v_c) (H v)_c)
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < OBS_THREADS / 32; ++w) t += red[w];
        double hp = 1.0;
        for (int k = 0; k < g.d; ++k) hp *= g.h[k];
        out[layer] = t * hp / (double)g.nf;
    }
}

int energy_impl(const dst_mesh *mesh, const double2 *psi, double *out, cudaStream_t s) {
    for (int k = 0; k < mesh->d; ++k)
        if (mesh->bc[k] != DST_BC_PERIODIC) {
            dst_internal_set_error_detail("dst_energy: every spatial axis must be periodic");
            return DST_ERR_ARG;
        }
    const int nc = mesh->nc;
    const int nx = (int)mesh->nu[0], ny = (int)mesh->nu[1], nz = (int)mesh->nu[2];
    if (nx > 4096 || ny > 4096 || nz > 4096) {
        dst_internal_set_error_detail("dst_energy: an axis longer than 4096 nodes");
        return DST_ERR_ARG;
    }
    // pass 1: (y, x) planes of every (layer, z); pass 2 (3+1): z lines of every (layer, fyx)
    SweepFft a1 = {}, a2 = {};
    a1.n1 = ny; a1.n2 = nx; a1.s1 = nx; a1.s2 = 1; a1.nbx = nz; a1.sbx = (int64_t)nx * ny;
    a1.ns_nodes = mesh->n_spatial; a1.nc = nc;
    dst_fft::radices(a1.n1, a1.rad1, a1.nrad1);
    dst_fft::radices(a1.n2, a1.rad2, a1.nrad2);
    const size_t limit = 200 * 1024;
    if (!dst_fft::choose_layout<double2>(a1, mesh->nt * nz, limit)) {
        dst_internal_set_error_detail("dst_energy: a layer plane too large for shared memory");
        return DST_ERR_ARG;
    }
    const int64_t nfyx = (int64_t)nx * ny;
    a2.n1 = nz; a2.n2 = 1; a2.s1 = nfyx; a2.s2 = 0; a2.nbx = (int)nfyx; a2.sbx = 1;
    a2.ns_nodes = nfyx * nz; a2.nc = nc;
    dst_fft::radices(a2.n1, a2.rad1, a2.nrad1);
    a2.nrad2 = 0;
    if (!dst_fft::choose_layout<double2>(a2, mesh->nt * nfyx, limit)) {
        dst_internal_set_error_detail("dst_energy: z axis too long for shared memory");
        return DST_ERR_ARG;
    }
    double2 *b1 = nullptr, *b2 = nullptr;
    const size_t bytes = sizeof(double2) * (size_t)mesh->n_unknowns;
    if (cudaMallocAsync(&b1, bytes, s) != cudaSuccess || (mesh->d == 3 && cudaMallocAsync(&b2, bytes, s) != cudaSuccess)) {
        cudaGetLastError();
        if (b1) cudaFreeAsync(b1, s);
        return DST_ERR_OOM;
    }
    static bool configured[64] = {};
    int dev = 0;
    int rc = DST_OK;
    if (cudaGetDevice(&dev) != cudaSuccess) rc = DST_ERR_CUDA;
    if (rc == DST_OK && (dev < 0 || dev >= 64 || !configured[dev])) {
        if (cudaFuncSetAttribute(dst_fft::fft_planes_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)limit) != cudaSuccess)
            rc = DST_ERR_CUDA;
        else if (dev >= 0 && dev < 64)
            configured[dev] = true;
    }
    if (rc == DST_OK) {
        const dim3 g1((unsigned)(mesh->nt * nz), (unsigned)(nc / a1.ncb));
        dst_fft::fft_planes_kernel<double2><<<g1, dst_fft::FFT_THREADS, dst_fft::fft_smem_bytes<double2>(a1), s>>>(
            a1, 0, psi, b1);
        if (mesh->d == 3) {
            const dim3 g2((unsigned)(mesh->nt * nfyx), (unsigned)(nc / a2.ncb));
            dst_fft::fft_planes_kernel<double2><<<g2, dst_fft::FFT_THREADS, dst_fft::fft_smem_bytes<double2>(a2), s>>>(
                a2, 0, b1, b2);
        }
        EGeo g;
        g.d = mesh->d; g.nc = nc; g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
        for (int k = 0; k < 3; ++k) g.h[k] = mesh->h[k];
        g.m = mesh->m;
        g.nf = mesh->n_spatial;
        energy_kernel<<<(unsigned)mesh->nt, OBS_THREADS, 0, s>>>(g, mesh->d == 3 ? b2 : b1, out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            dst_internal_set_cuda_error(e, "energy kernels", __FILE__, __LINE__);
            rc = DST_ERR_CUDA;
        }
    }
    cudaFreeAsync(b1, s);
    if (b2) cudaFreeAsync(b2, s);
    return rc;
}

}  // namespace

extern "C" int dst_energy(const dst_mesh *mesh, const void *psi, void *out, void *stream) {
    if (!mesh || !psi || !out || mesh->nt > 0x7fffffffLL) return DST_ERR_ARG;
    return energy_impl(mesh, (const double2 *)psi, (double *)out, (cudaStream_t)stream);
}

extern "C" int dst_observables(const dst_mesh *mesh, const void *psi, double x0, void *out, void *stream) {
    if (!mesh || !psi || !out || mesh->nt > 0x7fffffffLL) return DST_ERR_ARG;
    observables_kernel<<<(unsigned)mesh->nt, OBS_THREADS, 0, (cudaStream_t)stream>>>(
        geo(mesh, 0), geo(mesh, 1), geo(mesh, 2), mesh->d, mesh->nc, (const double2 *)psi, x0, (double *)out);
    DST_CUDA_TRY(cudaGetLastError());
    return DST_OK;
}
