// mc_sort.cuh -- keys-only LSD radix sort (mc_prims.cu) for the contraction's
// packed (block pair, weight) words.
#pragma once

#include "mc_internal.cuh"

namespace mc {

// Stable LSD sort of keysA[0..n) by the `bits` bits from bit `shift0` up
// (8-bit digits), ping-ponging with keysB; the bits below shift0 ride along
// untouched.  *in_b = the result is in keysB.  tmp: radix_tmp_words(n)
// words; scan_tmp: scan_tmp_words for 256 x ceil(n / 2048) entries.
int radix_sort_keys(u64 *keysA, u64 *keysB, i64 n, int shift0, int bits, u32 *tmp, int *scan_tmp, int *err,
                    bool *in_b, cudaStream_t s);

}  // namespace mc
