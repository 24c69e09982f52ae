// SLIC segmentation (the step before the method's Section III-A): the view
// records and the launch entry of k_slic.cu, kept apart from the hot path's
// declarations.
#pragma once
#include "lfd_internal.cuh"

namespace lfd {

// one view of a SLIC segmentation
struct SlicView {
    int W, H, GW, GH, fmt, pad;
    long long pitch;                 // bytes per image row
    const void *img;
    float4 *lab;                     // [W*H] CIELAB of the view (scratch)
    int *labels;                     // [W*H] output
    float *centres, *centres2;       // [GW*GH][5] {L, a, b, x, y} (scratch, ping-pong)
    unsigned long long *acc;         // [GW*GH][6] update sums {L, a, b (fixed point), x, y, count} (scratch)
};

// up to SLIC_BATCH views segmented by the same launches (blockIdx.y = view)
constexpr int SLIC_BATCH = 16;
struct SlicBatch {
    SlicView v[SLIC_BATCH];
    float wxy[SLIC_BATCH];                // (m / S)^2 of each view
    int n, max_px, max_cells, pad;
};

cudaError_t launch_slic(const SlicBatch &b, const float *const *centres_in, int iterations,
                        float *const *centres_out, cudaStream_t st);

}  // namespace lfd
