// Row stride of the weighted per-column root tables rdistq / rsigq: entry
// [t * stride + c] holds d(croot[c], t) and sigma from croot[c] to t. The
// row holds the group's columns only, rounded up to four (32-byte rows of
// 8-byte entries), so a vertex's entries for every column sit in the fewest
// sectors and the tables take n * stride entries of the n * 64 allocated.
#pragma once

namespace bcd {

__host__ __device__ __forceinline__ int wcols_stride(int ncols) { return (ncols + 3) & ~3; }

}  // namespace bcd
