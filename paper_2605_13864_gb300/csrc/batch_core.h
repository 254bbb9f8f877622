// batch_core.h -- the batch kernel's device tables and the helpers that
// build and launch them, shared by batch plans (batch.cu) and the serving
// engine (server.cu).  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/optigpu.h"

namespace optigpu {

// Device-side description of one instance.
struct BatchInst {
    const void *src;
    void *dst;
    int64_t rows;       // transpose rows, or the sum length n
    int64_t cols;       // transpose cols (1 for sums)
    int64_t first_item; // index of this instance's first work item
    int64_t aux;        // transpose: tiles per tile-row; sum: offset of its partials
    int32_t op;         // OPTIGPU_OP_TRANSPOSE / OPTIGPU_OP_REDUCE
    int32_t dtype;
    int32_t nitems;     // tiles or chunks
    int32_t vec_ok;     // sum: 16-byte aligned source
    int32_t th_log2;    // transpose tile height (source rows) = 1 << th_log2
    int32_t tw_log2;    // transpose tile width (source cols) = 1 << tw_log2
};

// Tile of a transpose instance: powers of two TH x TW with TH * TW <= area,
// square (sqrt(area) on a side) when both sides allow, otherwise as wide as
// the short side needs and as tall as the area allows, so skinny matrices
// still move a full tile per work item.
void batch_tile_shape(int64_t rows, int64_t cols, int area, int &th_log2, int &tw_log2);

// Host image of one batch: instances, the item -> instance map and totals.
struct BatchTables {
    std::vector<BatchInst> insts;
    std::vector<uint32_t> item_inst;
    int64_t items = 0;  // work items
    int64_t chunks = 0; // sum chunks (partial slots)
    int64_t bytes = 0;  // algorithmic bytes
};

// Byte offsets of one batch workspace: [queue][done counters][instances]
// [item map][partials].
struct BatchLayout {
    size_t off_queue, off_done, off_inst, off_items, off_part, total;
};

BatchLayout batch_layout(int64_t count, int64_t items, int64_t chunks);

// Checks one descriptor like the single calls do.
optigpu_status batch_validate(const optigpu_desc &d, int32_t index);

// Fills `t` for `count` validated descriptors; transposes are cut into tiles
// of at most `area` elements (batch_tile_shape).
optigpu_status batch_tables(const optigpu_desc *descs, int32_t count, int area, BatchTables &t);

// Transpose tile area of batch configuration `config`.
int batch_tile(int config);

// Enqueues the queue reset and the persistent batch kernel on `stream`.
// `clear_done` instances' completion counters are zeroed too (with the queue,
// which the layout places right before them): callers whose workspace held
// other tables before pass their instance count; plans, whose counters start
// at zero and are left at zero by every run, pass 0.  A negative `clear_done`
// means the caller has already zeroed the queue and the counters in work
// ordered before this launch on `stream`, so nothing is reset here.
// `sums_only` (every item is a sum chunk) selects the kernel form without a
// transpose tile, which fits more CTAs on an SM; results are the same.
optigpu_status batch_launch(int config, const BatchInst *d_insts, const uint32_t *d_item_inst, int64_t items,
                            unsigned long long *d_queue, unsigned *d_done, int64_t clear_done, void *d_partials,
                            int compensated, cudaStream_t stream, int *grid_out, bool sums_only);

} // namespace optigpu
