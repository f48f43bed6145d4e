// Library-internal access to a context (not part of the C ABI): the render
// server pre-sizes its slot contexts, bounds each batch's sort by an
// instance estimate, and reads each batch's status without a host
// synchronisation.
#pragma once

#include <cstdint>

#include "../../include/gs.h"

namespace gs {

// Grow every workspace of a fixed-capacity context to hold a batch of up to
// B views over a Gaussian set of this stride, `bins` tile bins, `pixels`
// pixels per channel and views of at most `view_tiles` tiles; later calls
// within those sizes allocate nothing.
gs_status ctx_reserve(gs_ctx* c, int64_t stride, int B, int64_t bins, int64_t pixels, int64_t view_tiles);

// Instance capacity of the following sorts: at most the context's fixed
// capacity (0 = the fixed capacity).  A smaller value shrinks the sort's
// grid; more instances than this set GS_ECAPACITY in the status word.
void ctx_set_batch_capacity(gs_ctx* c, int64_t cap);

// Forward-only context (render server): the forward pass records no
// contribution cells (no per-instance buffer, no zeroing) and gs_raster_bwd
// returns GS_ESTATE.
void ctx_set_forward_only(gs_ctx* c, bool on);

// Enqueue on the context's stream: copy the status word and the per-view
// instance counts of the last sort (B of them) into host memory (page-locked
// for an asynchronous copy), then clear the status word.
gs_status ctx_read_status_async(gs_ctx* c, int* status_host, uint64_t* view_totals_host, int B);

}  // namespace gs
