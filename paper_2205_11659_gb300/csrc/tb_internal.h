// tb_internal.h -- what the translation units of the library share: the
// phase-event hook, the look-back test hook and the workspace sizes of the
// operations that live in their own translation units.
#ifndef TB_INTERNAL_H
#define TB_INTERNAL_H

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "tb.h"

namespace tb_internal {

// Phase events: reset at the start of every public call, then one mark
// before each kernel and one after the last.
void phase_reset();
void phase_mark(cudaStream_t s);

// Element tile of the tree scans' depth pass that never publishes its
// look-back word (tb_debug_withhold_tile), or -1.
int withheld_tile();

// Scratch bytes of the tree scans (op TB_OP_TREE_SCAN or TB_OP_TREE_BACKWARD).
size_t tree_ws_bytes(int op, int64_t n);

// Scratch bytes of tb_open_positions.
size_t open_ws_bytes(int64_t n);

}  // namespace tb_internal

#endif  // TB_INTERNAL_H
