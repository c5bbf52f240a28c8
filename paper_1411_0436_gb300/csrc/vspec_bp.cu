// vspec_bp.cu — the persistent multi-bank kernel (vspec_bp.cuh) and the sizes
// its host side needs.
#include <cuda_runtime.h>

#define VSPEC_NO_PLAN_TABLES
#define VSPEC_DEFINE_BP_KERNEL
#include "vspec_bp.cuh"

const void *vspec_bp_kernel() { return (const void *)vspec::bp_kernel; }

// Dynamic shared memory of a bank's kernel-A ticket (form kBpColreg or
// kBpColdir, column length N2), 0 for a shape the kernel has no instance of.
size_t vspec_bp_smem_a(int form, int N2) {
    using namespace vspec;
    if (form == kBpColreg) {
        switch (N2) {
            case 2: return ColReg<2, 2>::smem;
            case 4: return ColReg<4, 4>::smem;
            case 8: return ColReg<8, 8>::smem;
            case 16: return ColReg<16, 16>::smem;
            case 32: return ColReg<32, 8>::smem;
            case 64: return ColReg<64, 8>::smem;
            case 128: return ColReg<128, 8>::smem;
        }
        return 0;
    }
    if (form == kBpColdir) {
        switch (N2) {
            case 2: return ColDir<2>::smem;
            case 4: return ColDir<4>::smem;
            case 8: return ColDir<8>::smem;
            case 16: return ColDir<16>::smem;
            case 32: return ColDir<32>::smem;
            case 64: return ColDir<64>::smem;
            case 128: return ColDir<128>::smem;
            case 256: return ColDir<256>::smem;
        }
    }
    return 0;
}

// Dynamic shared memory of a bank's kernel-B ticket: the 2048-point row
// body's four rows, or the one-row body's two groups.
size_t vspec_bp_smem_b(int form, int N1, int P) {
    using namespace vspec;
    if (form == kBpRowFir) return 2 * ((bp_rowfir_bytes(N1, P) + 15) & ~(size_t)15);
    return 4 * (size_t)kRow2048Stride * sizeof(P2);
}

// The kernel's bounds-check status word (debug builds), as vspec_ring_debug_flags.
cudaError_t vspec_bp_debug_flags(unsigned *flags, bool clear) {
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
