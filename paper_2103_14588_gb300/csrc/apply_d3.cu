// Operator apply and right-hand side instantiated for 3+1 dimensions (NC = 4).
// A general per-element potential takes the shared-memory kernel of
// apply_impl.cuh; x-only or vanishing potentials take the pipelined kernel of
// apply_pipe.cuh, or on meshes without open axes the z-column kernel of
// apply_zblk.cuh (tile variant 1).
#include "apply_zblk.cuh"

int dst_launch_apply_d3(const OpParams &p, int precision, const void *x, void *y, cudaStream_t s) {
    if (precision == DST_FP64) {
        if (p.vmode != 1) return dst::launch_apply_pipe<3, 4, double>(p, (const double2 *)x, (double2 *)y, s);
        return dst::launch_apply<3, 4, double>(p, (const double2 *)x, (double2 *)y, s);
    }
    if (p.vmode != 1) return dst::launch_apply_pipe<3, 4, float>(p, (const float2 *)x, (float2 *)y, s);
    return dst::launch_apply<3, 4, float>(p, (const float2 *)x, (float2 *)y, s);
}

int dst_launch_rhs_d3(const OpParams &p, const double2 *psi0, double2 *b, cudaStream_t s) {
    return dst::launch_rhs<3, 4>(p, psi0, b, s);
}
