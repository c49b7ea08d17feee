// Device-wide exclusive scans and ordered compactions used by graph set-up
// and query preparation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bcd.h"

namespace bcd {

// out[i] = sum of in[0..i) for i <= len (out has len + 1 entries).
// scratch may be NULL (then it is allocated for the call); otherwise it holds
// at least scan_scratch_len(len) entries.
bc_status scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t len, cudaStream_t s,
                             int64_t *scratch = nullptr, int64_t scratch_cap = 0);

// Ascending ids v in [0, n) whose mask passes the test: bit b of masks[v]
// when bit >= 0, masks[v] != 0 when bit < 0. out receives the ids, pos (may
// be NULL) receives out-index at each selected v, *d_count the number.
bc_status compact_mask(const uint64_t *masks, int bit, int64_t n, int32_t *out, int32_t *pos, int64_t *d_count,
                       cudaStream_t s, int64_t *scratch, int64_t scratch_cap);

int64_t scan_scratch_len(int64_t len);

}  // namespace bcd
