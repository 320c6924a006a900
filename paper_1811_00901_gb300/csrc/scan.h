// scan.h -- device exclusive prefix sum (internal).
#pragma once
#include "internal.h"

namespace si {
// out[k] = sum of in[0..k), k < n.  in == out is allowed.
si_status scan_exclusive(const int *in, int *out, int64_t n, cudaStream_t stream);
}  // namespace si
