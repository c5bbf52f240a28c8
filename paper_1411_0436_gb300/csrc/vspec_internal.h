// vspec_internal.h — host-side calls between the library's translation units
// (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "vspec.h"

// The persistent multi-bank launch (vspec_bp.cuh), implemented in vspec.cu.
// vspec_bp_supported: VSPEC_OK if plan p's calls can run as one of its banks
// (dual-pol, the register-column kernel A with 2048-point rows, or a one-row
// transform), else VSPEC_ERR_UNSUPPORTED with the reason in *why.
vspec_status vspec_bp_supported(const vspec_plan *p, const char **why);
// One launch over n plans' calls (n <= 16): ctl holds 2 + 2 n ints of control
// words, status the timeout flag; stall_bank >= 0 makes that bank's kernel-B
// tickets wait for a kernel-A ticket that never comes (failure tests).
vspec_status vspec_bp_execute(vspec_plan *const *plans, int n, const int8_t *const *d_in, const int *nspectra,
                              float *const *d_accum, int *ctl, int *status, int stall_bank, cudaStream_t st);
// Set the text vspec_last_error reports on this thread.
void vspec_set_last_error(const char *what);
