// Block-wide bitonic sorting of (key, configuration) records in shared
// memory.  Order: key ascending, then configuration ascending; the
// configuration integer makes every real record unique, which is the
// library's total order (energy, c).  Empty slots hold the largest key and
// c = ~0 and sort last.  All threads of the block must call these.
#pragma once

#include <cstdint>

namespace bf {

template <typename K>
__device__ __forceinline__ void cmp_swap(K* key, unsigned long long* cfg, int lo, int hi, bool ascending)
{
    K k0 = key[lo], k1 = key[hi];
    unsigned long long c0 = cfg[lo], c1 = cfg[hi];
    bool lo_greater = (k1 < k0) || (k1 == k0 && c1 < c0);
    if (lo_greater == ascending) {
        key[lo] = k1; key[hi] = k0;
        cfg[lo] = c1; cfg[hi] = c0;
    }
}

// Sort len (a power of two) records with the nt threads t = 0 .. nt-1 of a
// group that synchronises with sync().
template <typename K, typename Sync>
__device__ void group_sort(K* key, unsigned long long* cfg, int len, int t, int nt, Sync sync)
{
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            sync();
            for (int i = t; i < (len >> 1); i += nt) {
                int lo = ((i & -stride) << 1) + (i & (stride - 1));   // stride is a power of two
                cmp_swap(key, cfg, lo, lo + stride, (lo & size) == 0);
            }
        }
    }
    sync();
}

// Sort len (a power of two) records with the whole block.
template <typename K>
__device__ void block_sort(K* key, unsigned long long* cfg, int len)
{
    group_sort(key, cfg, len, (int)threadIdx.x, (int)blockDim.x, [] { __syncthreads(); });
}

// Merge two sorted halves [0, len/2) and [len/2, len) (len a power of two).
template <typename K>
__device__ void block_merge_halves(K* key, unsigned long long* cfg, int len)
{
    const int half = len >> 1;
    __syncthreads();
    // reverse the second half: the whole array becomes bitonic
    for (int i = threadIdx.x; i < (half >> 1); i += blockDim.x) {
        int a = half + i, b = len - 1 - i;
        K tk = key[a]; key[a] = key[b]; key[b] = tk;
        unsigned long long tc = cfg[a]; cfg[a] = cfg[b]; cfg[b] = tc;
    }
    for (int stride = half; stride > 0; stride >>= 1) {
        __syncthreads();
        for (int i = threadIdx.x; i < half; i += blockDim.x) {
            int lo = ((i & -stride) << 1) + (i & (stride - 1));   // stride is a power of two
            cmp_swap(key, cfg, lo, lo + stride, true);
        }
    }
    __syncthreads();
}

// Index of the first element with key > x in a sorted array (binary search).
template <typename K>
__device__ __forceinline__ int upper_bound_key(const K* key, int len, K x)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

}  // namespace bf
