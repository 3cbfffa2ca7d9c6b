// Warp tier: small and thin fronts (|N| <= 8 and |J| <= 32, or |J| <= 64 in
// the wider instance), one warp per task and right-hand side, the front
// staged in the warp's shared memory.
//
// Andersen, Dahl, Vandenberghe, "Logarithmic barriers for sparse matrix
// cones": the per-front formulas are those of the supernodal Algorithms
// 7.1-7.3 and of the block forms of Algorithms 5.1 and 5.2 (the same as the
// per-task and dense tiers); here every dense product is a warp-wide loop in
// which the 32 lanes take the output entries in turn.
//
// The front is held packed: entry (r, c), r >= c, of the lower triangle of
// the J x J front at  c*J - c*(c-1)/2 + (r - c).  The first n columns of this
// layout coincide with the front's N-part in the CSC value arrays, so loads
// and stores of values are contiguous copies.  Results other tiers read go
// to the front's workspace region in its dense layout (column-major, ld J):
// the update block (bottom-up passes) or the whole lower front (top-down).
#include <cuda_runtime.h>

#include <cstdint>

#include "chd_internal.h"
#include "front_views.cuh"

namespace chd_launch {
void count_launch();
}

// fronts with |J| <= 32: one warp per front, three per CTA
#define WT_NS w32
#define WT_J 32
#define WT_WPB 3
#define WT_TPF 32
#include "warp_tier_body.cuh"
#undef WT_NS
#undef WT_J
#undef WT_WPB
#undef WT_TPF

// chains of fronts with 32 < |J| <= 64 (bands of half-bandwidth up to 63):
// eight warps (one CTA) per front, which shortens the serial chain
#define WT_NS w64
#define WT_J 64
#define WT_WPB 1
#define WT_TPF 256
#include "warp_tier_body.cuh"
#undef WT_NS
#undef WT_J
#undef WT_WPB
#undef WT_TPF
