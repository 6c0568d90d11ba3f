// tb_internal.h -- what the translation units of the library share: the
// matching pass as a callable step, the phase-event hook and the tree-scan
// workspace size.
#ifndef TB_INTERNAL_H
#define TB_INTERNAL_H

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "tb.h"

namespace tb_internal {

// Scratch bytes of the matching pass over n elements.
size_t match_ws_bytes(int64_t n);

// The matching pass of tb_match_parens (status cleared first), recording
// phase events like the public call.
tb_status run_match(const uint8_t* kind, int64_t n, int32_t* parent, int32_t* match, void* ws,
                    size_t ws_bytes, int32_t* d_status, cudaStream_t s);

// Phase events: reset at the start of every public call, then one mark
// before each kernel and one after the last.
void phase_reset();
void phase_mark(cudaStream_t s);

// Scratch bytes of the tree scans (op TB_OP_TREE_SCAN or TB_OP_TREE_BACKWARD).
size_t tree_ws_bytes(int op, int64_t n);

}  // namespace tb_internal

#endif  // TB_INTERNAL_H
