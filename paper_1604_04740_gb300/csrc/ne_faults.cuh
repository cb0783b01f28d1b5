// Transient-fault hook shared by the fused epilogues: the faults of the fault
// model of Sec. I (one stream's result of the operation corrupted) are XORed
// into the words delta right before the extraction, so the check of Eq. 24
// and the extraction of Eq. 17-20 see them exactly as they would see a fault
// of the operation itself.  Lists are sorted by flat output position.
#pragma once

#include "ne_common.cuh"

namespace ne {

// first index f in [lo, hi) with pos[f] >= key (pos sorted ascending)
__device__ __forceinline__ int64_t fault_lower_bound(const int64_t* pos, int64_t lo, int64_t hi, int64_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pos[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// XOR every listed fault at flat position key on stream m into v; [f0, f1)
// is a range of the list that contains every entry at key
__device__ __forceinline__ int64_t apply_faults(int64_t v, const int64_t* pos, const int32_t* stream,
                                                const int32_t* bit, int64_t f0, int64_t f1, int64_t key, int m) {
    for (int64_t f = fault_lower_bound(pos, f0, f1, key); f < f1 && pos[f] == key; f++)
        if (stream[f] == m) v ^= (int64_t)(1ull << (bit[f] & 63));
    return v;
}

}  // namespace ne
