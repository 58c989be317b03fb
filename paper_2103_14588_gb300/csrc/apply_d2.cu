// Operator apply and right-hand side instantiated for 2+1 dimensions (NC = 2).
// A general per-element potential takes the shared-memory kernel of
// apply_impl.cuh; x-only or vanishing potentials take the pipelined kernel of
// apply_pipe.cuh, in FP32 on meshes without an open axis its two-threads-per-
// node form (apply_pipe2h.cuh).
#include "apply_pipe2h.cuh"

int dst_launch_apply_d2(const OpParams &p, int precision, const void *x, void *y, cudaStream_t s) {
    if (precision == DST_FP64) {
        if (p.vmode != 1) return dst::launch_apply_pipe<2, 2, double>(p, (const double2 *)x, (double2 *)y, s);
        return dst::launch_apply<2, 2, double>(p, (const double2 *)x, (double2 *)y, s);
    }
    if (p.vmode != 1) {
        if (p.ax[0].bc != DST_BC_OPEN && p.ax[1].bc != DST_BC_OPEN) {
            const int tv = p.tile_variant[DST_FP32];
            if (tv == 1) return dst::launch_apply_pipe2h<1>(p, (const float2 *)x, (float2 *)y, s);
            if (tv == 2) return dst::launch_apply_pipe2h<2>(p, (const float2 *)x, (float2 *)y, s);
            return dst::launch_apply_pipe2h<0>(p, (const float2 *)x, (float2 *)y, s);
        }
        return dst::launch_apply_pipe<2, 2, float>(p, (const float2 *)x, (float2 *)y, s);
    }
    return dst::launch_apply<2, 2, float>(p, (const float2 *)x, (float2 *)y, s);
}

int dst_launch_rhs_d2(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s) {
    return dst::launch_rhs<2, 2>(p, psi0, b, s);
}
