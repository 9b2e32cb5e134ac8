// Device-side tables and launchers of the batched step (lbm_batch.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// One case of a batch, as the kernels see it (device table).
struct BatchCase {
    Geometry geo;     // lattice, padding and pitch of this case's planes
    long long off;    // element offset of the case's 18 planes in each arena buffer
    int ntx;          // tiles across x for the tile shape in use
    int ntiles;
    float rest_sum;   // sum of the nine f rest populations (shifted formats; else 0)
    int pad;
};

struct BatchItem {
    int c;     // case
    int tile;  // tile index within the case, row-major over (ntx, nty)
};

struct BatchLaunch {
    const BatchItem* items;
    int nitems;
    const BatchCase* cases;
    const KC<float>* kcs;
    const CUtensorMap* maps;  // [case][buffer][f, g] for the tile shape in use
    float* partials;          // [nitems][8]
    int* status;
    int sms;
    double* steps;            // steps the batch has executed (device; keys stochastic rounding)
    unsigned* done;           // blocks of the current launch that have finished
    int rounding;             // 16-bit storage: 0 nearest, 1 stochastic
    unsigned long long tile_wait_ns;  // bound on each wait for an item's copies; 0: no waiting
};

void batch_tile(int storage, int variant, int* bx, int* by);
cudaError_t batch_prepare(int storage);
cudaError_t launch_batch_step(int storage, int variant, const BatchLaunch& B, int from, void* out, cudaStream_t s);
cudaError_t launch_batch_case_record(const BatchLaunch& B, int c, double* out, cudaStream_t s);

}  // namespace lbm
