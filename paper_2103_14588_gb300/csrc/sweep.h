// Crank-Nicolson sweep preconditioner (sweep.cu): plan, scratch and application.
#pragma once

#include "internal.h"

// FFT of the planes of periodic axes: plane b covers the nodes
// base(b) + i1 * s1 + i2 * s2 (i1 < n1, i2 < n2), base(b) = (b / nbx) * ns_nodes + (b % nbx) * sbx.
struct SweepFft {
    int n1, n2;                 // outer and inner FFT lengths (1: no such axis)
    int64_t s1, s2;             // node strides of the two FFT dimensions
    int nbx;                    // batches per layer (x nodes in banded mode, else 1)
    int64_t sbx;                // node stride between the batches of one layer
    int64_t ns_nodes;           // nodes of one layer
    int nc, ncb;                // spinor components, components per CTA
    int rad1[32], rad2[32];     // Stockham radices of each length
    int nrad1, nrad2;
    int pingpong;               // 1: CTA-wide stages with a second plane buffer
};

struct SweepGeom {
    int d, nc;
    int64_t nt;
    double ht, m, V0;           // V0: the constant potential of a spectral mesh
    double h[3];
    int nx;                     // unknown x nodes (banded mode)
    int n1, n2;                 // frequency grid (outer, inner); nf = n1 * n2
    int ax1, ax2;               // physical axis of each frequency dimension (-1: none)
};

struct SweepPlan {
    SweepGeom g;
    SweepFft fft;
    bool banded, has_fft, vx;
    int64_t nb;                 // FFT planes
    size_t fft_smem;
    size_t table_bytes;         // banded: block Thomas factors
    int march_threads;
    size_t march_smem;
    // set by dst_sweep_setup inside the caller's scratch
    float2 *work;
    float2 *table;
    double *dvx;
};

// DST_OK or DST_ERR_ARG (with a detail) for meshes the sweep does not cover.
int dst_sweep_plan(const dst_mesh *mesh, SweepPlan &p);
// Device scratch the sweep needs: one FP32 vector, the factors, the potential.
size_t dst_sweep_scratch_bytes(const SweepPlan &p, int64_t n_unknowns);
// Carve the scratch and compute the banded factors (enqueued on s).
int dst_sweep_setup(const dst_mesh *mesh, SweepPlan &p, void *scratch, cudaStream_t s);
// z = B^-1 S^-1 v on FP32 vectors (enqueued on s); v and z distinct.
int dst_sweep_apply(const SweepPlan &p, int64_t n_unknowns, const float2 *v, float2 *z, cudaStream_t s);
