// Global selection (steps A4 and A5).
//
// The enumeration kernel leaves one sorted list of at most `cap` records
// per block (records: quantised energy, configuration).  merge_kernel merges
// lists pairwise (a tree of launches, the paper's running merge of a chunk's
// lowest states with the global record, Algorithm 1), absorb_kernel folds
// the spill area into the lists, and the finalize kernels write the S
// lowest records: exact integers directly, float instances after an FP64
// re-evaluation of Eq. (1) (Sec. 2) and an exact reselection by (E, c).
//
// Keep rule after every merge (sorted records, S-th record energy K):
//   integer instances (W = 0): the first S records;
//   float instances: every record with E <= K + W, at least the first S.
// A record dropped by this rule cannot be among the final S lowest: the
// S records before it are real configurations with lower quantised keys.
#include <cfloat>
#include <climits>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kMergeThreads = 512;

// keep count of a sorted array of `len` records with `valid` real ones
__device__ int keep_count(const int* E, int len, int valid, int S, int W, int cap, WsHeader* hdr)
{
    if (valid < S) return valid;
    const int K = E[S - 1];
    if (W == 0) return S;
    long long lim = (long long)K + W;
    int keep = upper_bound_key(E, len, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
    if (keep > valid) keep = valid;
    if (keep > cap) {
        keep = cap;
        atomicOr(&hdr->status, kErrWindow);
    }
    return keep;
}

__global__ void __launch_bounds__(kMergeThreads) merge_kernel(const int* inE, const unsigned long long* inC, int nin,
                                                              int* outE, unsigned long long* outC, int cap, int S,
                                                              int W, WsHeader* hdr, const int* Wp)
{
    if (Wp) W = *Wp;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);
    int* E = reinterpret_cast<int*>(C + 2 * cap);
    __shared__ int s_keep;
    const int a = 2 * blockIdx.x, b = a + 1;
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        E[i] = inE[(size_t)a * cap + i];
        C[i] = inC[(size_t)a * cap + i];
        E[cap + i] = b < nin ? inE[(size_t)b * cap + i] : kEmptyE;
        C[cap + i] = b < nin ? inC[(size_t)b * cap + i] : kEmptyC;
    }
    block_merge_halves(E, C, 2 * cap);
    if (threadIdx.x == 0) {
        int valid = upper_bound_key(E, 2 * cap, INT_MAX - 1);
        s_keep = keep_count(E, 2 * cap, valid, S, W, cap, hdr);
    }
    __syncthreads();
    const int keep = s_keep;
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        outE[(size_t)blockIdx.x * cap + i] = i < keep ? E[i] : kEmptyE;
        outC[(size_t)blockIdx.x * cap + i] = i < keep ? C[i] : kEmptyC;
    }
}

__global__ void __launch_bounds__(kMergeThreads) absorb_kernel(int* LE, unsigned long long* LC, int nlists, int cap,
                                                               int S, int W, const int* spE,
                                                               const unsigned long long* spC, unsigned spill_cap,
                                                               WsHeader* hdr, const int* Wp)
{
    if (Wp) W = *Wp;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);
    int* E = reinterpret_cast<int*>(C + 2 * cap);
    __shared__ int s_keep;
    unsigned count = *(volatile unsigned*)&hdr->spill_count;
    if (count > spill_cap) count = spill_cap;
    const size_t me = (size_t)blockIdx.x * cap;
    if ((unsigned long long)blockIdx.x * cap >= count) return;   // uniform over the block
    for (int i = threadIdx.x; i < cap; i += blockDim.x) { E[i] = LE[me + i]; C[i] = LC[me + i]; }
    for (unsigned long long ch = blockIdx.x; ch * cap < count; ch += nlists) {
        const unsigned long long off = ch * cap;
        __syncthreads();
        for (int i = threadIdx.x; i < cap; i += blockDim.x) {
            bool ok = off + i < count;
            E[cap + i] = ok ? spE[off + i] : kEmptyE;
            C[cap + i] = ok ? spC[off + i] : kEmptyC;
        }
        // sort the chunk in place (upper half), then merge with the list (lower half)
        __syncthreads();
        block_sort(E + cap, C + cap, cap);
        block_merge_halves(E, C, 2 * cap);
        if (threadIdx.x == 0) {
            int valid = upper_bound_key(E, 2 * cap, INT_MAX - 1);
            s_keep = keep_count(E, 2 * cap, valid, S, W, cap, hdr);
        }
        __syncthreads();
        const int keep = s_keep;
        for (int i = threadIdx.x; i < cap; i += blockDim.x)
            if (i >= keep) { E[i] = kEmptyE; C[i] = kEmptyC; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cap; i += blockDim.x) { LE[me + i] = E[i]; LC[me + i] = C[i]; }
}

// ---- final selection -------------------------------------------------------

// Zero-field searches walk the half space with spin n-1 at -1: the sorted list holds its lowest
// records, and with their mirrors c ^ (2^n - 1), of the same energy, they contain the S lowest of
// the whole space (a mirror's original has the smaller c, so it comes first in (E, c) order).
// Within one energy the half-space records come first in increasing c, then the mirrors in the
// reverse order.  One thread writes the S outputs; key_at(t) is the t-th sorted key, and real
// records end at the first empty one.
template <typename KeyAt, typename Empty, typename Write>
__device__ void emit_with_mirrors(int len, int S, int n, KeyAt key_at, Empty empty, Write write)
{
    const unsigned long long mirror = n >= 64 ? ~0ull : (1ull << n) - 1ull;
    int keep = 0;
    while (keep < len && !empty(keep)) keep++;
    int out = 0, i = 0;
    while (out < S && i < keep) {
        int j = i + 1;
        while (j < keep && key_at(j) == key_at(i)) j++;
        for (int t = i; t < j && out < S; t++) write(out++, t, 0ull);
        for (int t = j - 1; t >= i && out < S; t--) write(out++, t, mirror);
        i = j;
    }
    for (; out < S; out++) write(out, -1, 0ull);
}

__global__ void __launch_bounds__(256) finalize_int_kernel(const int* E, const unsigned long long* C, int S, int q,
                                                           const int* qp, const int* z2p, int n, int len,
                                                           long long* energies, unsigned long long* states)
{
    if (qp) q = *qp;
    if (z2p && *z2p) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            emit_with_mirrors(len, S, n, [&](int t) { return E[t]; }, [&](int t) { return E[t] == kEmptyE; },
                              [&](int k, int t, unsigned long long x) {
                                  energies[k] = t >= 0 ? (long long)(E[t] >> q) : LLONG_MAX;
                                  states[k] = t >= 0 ? C[t] ^ x : kEmptyC;
                              });
        return;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
        energies[k] = (long long)(E[k] >> q);   // E_q = E * 2^q exactly for integer instances
        states[k] = C[k];
    }
}

__device__ __forceinline__ double load_value(const void* p, int dtype, size_t idx)
{
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

// Eq. (1) in FP64, one warp per record: lane i holds s_i (h_i + sum_{j>i} J_ij s_j)
__global__ void __launch_bounds__(256) rescore_kernel(const int* E, const unsigned long long* C, int cap, int n,
                                                      int dtype, const void* J, const void* h, double* out)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < cap; r += nwarps) {
        if (E[r] == kEmptyE) {
            if (lane == 0) out[r] = DBL_MAX;
            continue;
        }
        const unsigned long long c = C[r];
        double part = 0.0;
        for (int i = lane; i < n; i += 32) {
            double row = load_value(h, dtype, i);
            for (int j = i + 1; j < n; j++) {
                double v = load_value(J, dtype, (size_t)i * n + j);
                row += ((c >> j) & 1ull) ? v : -v;
            }
            part += ((c >> i) & 1ull) ? row : -row;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) out[r] = part;
    }
}

__global__ void __launch_bounds__(kMergeThreads) finalize_float_kernel(const unsigned long long* C, const double* E64,
                                                                       int cap, int S, const int* z2p, int n,
                                                                       double* energies, unsigned long long* states)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* cfg = reinterpret_cast<unsigned long long*>(smem);
    double* key = reinterpret_cast<double*>(cfg + cap);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        key[i] = E64[i];
        cfg[i] = C[i];
    }
    block_sort(key, cfg, cap);
    if (z2p && *z2p) {
        if (threadIdx.x == 0)
            emit_with_mirrors(cap, S, n, [&](int t) { return key[t]; }, [&](int t) { return cfg[t] == kEmptyC; },
                              [&](int k, int t, unsigned long long x) {
                                  energies[k] = t >= 0 ? key[t] : DBL_MAX;
                                  states[k] = t >= 0 ? cfg[t] ^ x : kEmptyC;
                              });
        return;
    }
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        energies[k] = key[k];
        states[k] = cfg[k];
    }
}

}  // namespace

cudaError_t launch_merge_round(const int* inE, const unsigned long long* inC, int nin, int* outE,
                               unsigned long long* outC, int cap, int S, int W, WsHeader* hdr, cudaStream_t s,
                               const int* Wp)
{
    size_t smem = (size_t)2 * cap * 12;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(merge_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    merge_kernel<<<(nin + 1) / 2, kMergeThreads, smem, s>>>(inE, inC, nin, outE, outC, cap, S, W, hdr, Wp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_absorb_spill(int* E, unsigned long long* C, int nlists, int cap, int S, int W, const int* spill_E,
                                const unsigned long long* spill_C, unsigned spill_cap, WsHeader* hdr,
                                cudaStream_t s, const int* Wp)
{
    size_t smem = (size_t)2 * cap * 12;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(absorb_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    absorb_kernel<<<nlists, kMergeThreads, smem, s>>>(E, C, nlists, cap, S, W, spill_E, spill_C, spill_cap, hdr, Wp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const int* E, const unsigned long long* C, int cap, int S, int n, int dtype, int q,
                            const void* J, const void* h, double* rescore, void* energies,
                            unsigned long long* states, WsHeader* hdr, cudaStream_t s, const int* qp,
                            const int* z2p)
{
    (void)hdr;
    if (dtype == 0) {
        finalize_int_kernel<<<(S + 255) / 256, 256, 0, s>>>(E, C, S, q, qp, z2p, n, cap,
                                                            static_cast<long long*>(energies), states);
        count_launches(1);
        return cudaGetLastError();
    }
    rescore_kernel<<<(cap + 7) / 8, 256, 0, s>>>(E, C, cap, n, dtype, J, h, rescore);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t smem = (size_t)cap * 16;
    e = ensure_smem(reinterpret_cast<const void*>(finalize_float_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    finalize_float_kernel<<<1, kMergeThreads, smem, s>>>(C, rescore, cap, S, z2p, n, static_cast<double*>(energies),
                                                         states);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
