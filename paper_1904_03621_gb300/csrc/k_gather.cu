// Final selection in one launch (steps A4 and A5 of one search).
//
// After the enumeration every block of the walk has left a sorted list of
// its lowest records (quantised energy, configuration), and records that did
// not fit a block's buffer sit unsorted in the spill area.  The global
// threshold tau (the lowest S-th energy any block published) bounds the
// S-th lowest quantised energy of the whole space from above, so only
// records with E <= tau + W can belong to the answer, W being the float
// window of the fixed-point screen (0 for integer instances).  One block:
//   1. the length of every list's prefix with E <= tau + W (binary search),
//      and their exclusive scan;
//   2. those records, then the spill records with E <= tau + W, are appended
//      to a shared-memory buffer in chunks; after every chunk the buffer is
//      sorted by (E, c) and cut to the first S records plus, for float
//      instances, every record within W of the S-th (the keep rule of the
//      pairwise merges, Algorithm 1's running selection);
//   3. integer instances write E_q / 2^q and c of the first S records; float
//      instances re-evaluate Eq. (1) of every kept record in FP64, sort by
//      (E, c) and write the first S.
// In the common case the filtered records fit one chunk, so the whole
// selection is one launch instead of a spill merge, log2(lists) merge rounds
// and two finalising kernels.
#include <cfloat>
#include <climits>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kGatherThreads = 1024;

__device__ __forceinline__ double load_value(const void* p, int dtype, size_t idx)
{
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

// Sort the first `count` records of the buffer (padded to a power of two) and return how many
// the keep rule retains.
__device__ int sort_keep(int* E, unsigned long long* C, int count, int S, int W, int cap, WsHeader* hdr,
                         int* s_keep)
{
    int len = 64;
    while (len < count) len <<= 1;
    for (int i = count + (int)threadIdx.x; i < len; i += blockDim.x) {
        E[i] = kEmptyE;
        C[i] = kEmptyC;
    }
    block_sort(E, C, len);
    if (threadIdx.x == 0) {
        const int valid = upper_bound_key(E, len, INT_MAX - 1);
        int keep = valid;
        if (valid >= S) {
            keep = S;
            if (W > 0) {
                const long long lim = (long long)E[S - 1] + W;
                keep = upper_bound_key(E, len, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
                if (keep > valid) keep = valid;
            }
        }
        if (keep > cap) {
            keep = cap;
            atomicOr(&hdr->status, kErrWindow);
        }
        *s_keep = keep;
    }
    __syncthreads();
    return *s_keep;
}

__global__ void __launch_bounds__(kGatherThreads, 1) gather_final_kernel(const GatherParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);   // buf
    double* key = reinterpret_cast<double*>(C + p.buf);                     // cap
    unsigned long long* cf = reinterpret_cast<unsigned long long*>(key + p.cap);   // cap
    double* Jd = reinterpret_cast<double*>(cf + p.cap);                     // n*n (float instances)
    double* hd = Jd + p.n * p.n;                                            // n
    int* E = reinterpret_cast<int*>(hd + p.n);                              // buf
    int* pre = E + p.buf;                                                   // nlists + 1
    __shared__ int s_keep, s_wsum[kGatherThreads / 32];
    __shared__ unsigned s_fill;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = p.S, cap = p.cap;
    const int W = *p.Wp;
    const long long lim64 = (long long)(*(volatile int*)&p.hdr->tau) + W;
    const int lim = lim64 > INT_MAX - 1 ? INT_MAX - 1 : (int)lim64;

    // 1. prefix lengths of the lists and their exclusive scan (nlists <= blockDim.x)
    int len = 0;
    if (tid < p.nlists) len = upper_bound_key(p.list_E + (size_t)tid * cap, cap, lim);
    int v = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = s_wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_wsum[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += s_wsum[warp - 1];
    if (tid < p.nlists) pre[tid + 1] = v;       // inclusive sums
    if (tid == 0) pre[0] = 0;
    __syncthreads();
    const int total = pre[p.nlists];

    // 2. append in chunks, sort, keep
    const int chunk = p.buf - cap;
    int kept = 0;
    for (int r0 = 0; r0 < total; r0 += chunk) {
        const int m = min(chunk, total - r0);
        for (int i = tid; i < m; i += blockDim.x) {
            const int r = r0 + i;
            int lo = 0, hi = p.nlists;                 // list l holds records [pre[l], pre[l + 1])
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pre[mid] <= r) lo = mid; else hi = mid;
            }
            const size_t at = (size_t)lo * cap + (size_t)(r - pre[lo]);
            E[kept + i] = p.list_E[at];
            C[kept + i] = p.list_C[at];
        }
        __syncthreads();
        kept = sort_keep(E, C, kept + m, S, W, cap, p.hdr, &s_keep);
    }
    unsigned nsp = *(volatile unsigned*)&p.hdr->spill_count;
    if (nsp > p.spill_cap) nsp = p.spill_cap;
    for (unsigned s0 = 0; s0 < nsp; s0 += (unsigned)chunk) {
        if (tid == 0) s_fill = 0u;
        __syncthreads();
        const unsigned m = min((unsigned)chunk, nsp - s0);
        for (unsigned i = tid; i < m; i += blockDim.x) {
            const int e = p.spill_E[s0 + i];
            if (e <= lim) {
                const unsigned slot = atomicAdd(&s_fill, 1u);
                E[kept + slot] = e;
                C[kept + slot] = p.spill_C[s0 + i];
            }
        }
        __syncthreads();
        const int got = (int)s_fill;
        if (got > 0) kept = sort_keep(E, C, kept + got, S, W, cap, p.hdr, &s_keep);
    }

    // 3. outputs
    if (p.dtype == 0) {
        const int q = *p.qp;
        for (int k = tid; k < S; k += blockDim.x) {
            static_cast<long long*>(p.energies)[k] = k < kept ? (long long)(E[k] >> q) : LLONG_MAX;
            p.states[k] = k < kept ? C[k] : kEmptyC;
        }
        return;
    }
    // float: Eq. (1) in FP64 for every kept record, one warp per record (lane i holds
    // s_i (h_i + sum_{j>i} J_ij s_j)), with J and h staged in shared memory, then the exact
    // reselection by (E, c)
    for (int idx = tid; idx < p.n * p.n; idx += blockDim.x) Jd[idx] = load_value(p.J, p.dtype, idx);
    for (int i = tid; i < p.n; i += blockDim.x) hd[i] = load_value(p.h, p.dtype, i);
    __syncthreads();
    int flen = 1;
    while (flen < kept || flen < 2) flen <<= 1;
    for (int r = warp; r < flen; r += kGatherThreads / 32) {
        if (r >= kept) {
            if (lane == 0) { key[r] = DBL_MAX; cf[r] = kEmptyC; }
            continue;
        }
        const unsigned long long c = C[r];
        double part = 0.0;
        for (int i = lane; i < p.n; i += 32) {
            double row = hd[i];
            const double* Ji = Jd + i * p.n;
            for (int j = i + 1; j < p.n; j++) row += ((c >> j) & 1ull) ? Ji[j] : -Ji[j];
            part += ((c >> i) & 1ull) ? row : -row;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) { key[r] = part; cf[r] = c; }
    }
    __syncthreads();
    block_sort(key, cf, flen);
    for (int k = tid; k < S; k += blockDim.x) {
        static_cast<double*>(p.energies)[k] = key[k];
        p.states[k] = cf[k];
    }
}

}  // namespace

size_t gather_smem_bytes(int nlists, int cap, int buf, int n)
{
    return (size_t)buf * 12 + (size_t)cap * 16 + (size_t)(n * n + n) * 8 + (size_t)(nlists + 1) * 4;
}

int gather_buffer(int cap) { return cap * 2 > 4096 ? cap * 2 : 4096; }

cudaError_t launch_gather_final(const GatherParams& p, cudaStream_t s)
{
    if (p.nlists < 1 || p.nlists > kMaxGatherLists || p.buf < 2 * p.cap) return cudaErrorInvalidValue;
    const size_t smem = gather_smem_bytes(p.nlists, p.cap, p.buf, p.n);
    cudaError_t e = cudaFuncSetAttribute(gather_final_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gather_final_kernel<<<1, kGatherThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
