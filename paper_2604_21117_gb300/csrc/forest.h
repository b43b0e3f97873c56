// Internal interface of the multi-tree launch, shared by forest.cu and the
// serving loop (server.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bt_internal.h"

namespace btgb {

// One tree of a forest as the batching kernel sees it: the tree (with the
// top levels this forest pins), its optional learned model and the launch
// settings taken from the tree's tuning or the forest's overrides.
struct ForestTree {
    DevTree t;
    ModelDev md;       // kind kModelNone: plain descent only
    int lq;            // queries per lane: 1 (32-query chunks) or 2 (64-query chunks)
    int staged;        // levels below the pinned ones: warp-staged node blocks (1) or per-lane reads through L1 (0)
    uint32_t pin_off;  // byte offset of the pinned levels in the block's shared memory
    uint32_t pad_;
};

// Completion signal of a launch, for a host that polls memory instead of
// events: every block adds one to *counter after a system-scope fence; the
// last block to arrive resets the counter and stores `seq` to *flag
// (host-mapped memory).  counter == nullptr: no signal.
struct ForestDone {
    unsigned int *counter;
    unsigned long long *flag;
    unsigned long long seq;
};

// Launch the batching kernel over a work list.  chunk_start: the work
// list's chunk offsets (nb + 1 entries, device-visible) when the host
// computed them (forest_chunks; host_chunks = their total, which sizes the
// grid), else nullptr and plan_ws (nb + 1 words of device memory) receives
// them from the plan kernel.  batches, chunk_start, q and the outputs may be
// host-mapped memory.  warps: 1..16.
cudaError_t forest_run(const bt_forest *f, const bt_batch_desc *batches, uint32_t nb, const uint32_t *chunk_start,
                       uint32_t host_chunks, uint32_t *plan_ws, const void *q, uint64_t nq, void *out_v,
                       uint8_t *out_f, uint32_t warps, cudaStream_t s, ForestDone done);

// Host-side plan: chunk offsets of a work list (nb + 1 entries), with the
// forest's chunk width per tree.
void forest_chunks(const bt_forest *f, const bt_batch_desc *batches, uint32_t nb, uint32_t *chunk_start);

uint32_t forest_default_warps(const bt_forest *f);

}  // namespace btgb
