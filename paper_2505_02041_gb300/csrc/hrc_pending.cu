// hrc_pending.cu -- entry points whose kernels are not written yet; each
// reports HRC_ESTATE so that callers see a clear error.
#include "hrc.h"

extern "C" {
hrc_status hrc_create_batched(int, const int *, const int *, int, int, hrc_ctx **out) { if (out) *out = 0; return HRC_ESTATE; }
hrc_status hrc_scene_offsets(const hrc_ctx *, long long *, long long *) { return HRC_ESTATE; }
hrc_status hrc_fluence_batched(hrc_ctx *, const float *, const float *, float *) { return HRC_ESTATE; }
hrc_status hrc_fluence_backward_batched(hrc_ctx *, const float *, float *, float *) { return HRC_ESTATE; }
}
