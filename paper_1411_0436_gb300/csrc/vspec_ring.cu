// vspec_ring.cu — instances of the persistent ring kernel (vspec_ring.cuh),
// one per column length of the register-column kernel A.
#include <cuda_runtime.h>

#define VSPEC_NO_PLAN_TABLES
#include "vspec_ring.cuh"

// The ring kernel for N2-point columns (2 .. 128), its dynamic shared memory
// in *smem; nullptr for other lengths.
const void *vspec_pick_kernel_ring(int N2, size_t *smem) {
    using namespace vspec;
    switch (N2) {
        case 2: *smem = RingShape<2, 2>::smem; return (const void *)ring_kernel<2, 2>;
        case 4: *smem = RingShape<4, 4>::smem; return (const void *)ring_kernel<4, 4>;
        case 8: *smem = RingShape<8, 8>::smem; return (const void *)ring_kernel<8, 8>;
        case 16: *smem = RingShape<16, 16>::smem; return (const void *)ring_kernel<16, 16>;
        case 32: *smem = RingShape<32, 8>::smem; return (const void *)ring_kernel<32, 8>;
        case 64: *smem = RingShape<64, 8>::smem; return (const void *)ring_kernel<64, 8>;
        case 128: *smem = RingShape<128, 8>::smem; return (const void *)ring_kernel<128, 8>;
    }
    return nullptr;
}

// The ring kernels' bounds-check status word (debug builds): read into
// *flags, cleared if `clear`.
cudaError_t vspec_ring_debug_flags(unsigned *flags, bool clear) {
#ifdef VSPEC_DEBUG
    cudaError_t e = cudaMemcpyFromSymbol(flags, vspec::g_debug_flags, sizeof(unsigned));
    if (e != cudaSuccess || !clear) return e;
    const unsigned zero = 0;
    return cudaMemcpyToSymbol(vspec::g_debug_flags, &zero, sizeof(unsigned));
#else
    *flags = 0;
    (void)clear;
    return cudaSuccess;
#endif
}
