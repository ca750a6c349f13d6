// plan.cuh -- plan construction in two steps, shared by the C API and the
// request server: the host-side layout (argument checks, launch geometry and
// the size of the workspace; no device memory, no synchronisation) and the
// device allocation.  The server sizes a plan with the first step and only
// allocates once the plan fits its memory budget.
#pragma once

#include "common.cuh"

namespace fp {

// Validates the arguments and lays the plan out.  On FPSNR_OK *out is a plan
// whose slab_bytes is the device workspace it needs and which owns no device
// memory yet (release it with delete, or pass it to plan_allocate).  Errors:
// FPSNR_EINVAL (arguments), FPSNR_ENOMEM (host memory), FPSNR_ECUDA (device
// attributes); *out is then null.
int plan_layout(fpsnr_plan_s** out, int ndim, const uint64_t* dims, double target_psnr_db,
                const fpsnr_opts* opts);

// Allocates and initialises the workspace of a plan from plan_layout
// (synchronises the device once).  FPSNR_OK, or FPSNR_ENOMEM / FPSNR_ECUDA
// after deleting the plan.
int plan_allocate(fpsnr_plan_s* p);

}  // namespace fp
