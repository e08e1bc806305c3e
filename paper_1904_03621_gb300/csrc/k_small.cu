// Small search spaces (2^13 .. 2^20 configurations): exact enumeration without a walk.
//
// For spaces this small the walk of k_gray.cu has too little work to fill the GPU, and its
// first threshold (a sample of up to 2^20 configurations evaluated by the O(n^2)
// definition, then merged) costs more than the whole space.  small_enum_kernel: block b
// enumerates the 8192 configurations whose bits [13, free) equal b, in exact int32 fixed
// point.  The block evaluates its base configuration (13 low spins at -1) and the fields of
// those spins by the definition (Eq. (1)); thread t reaches its start (spins 4..12 = the bits
// of t) by flipping those spins one at a time (E += 2 f_v, the current field of spin v), then
// walks spins 0..3 in reflected Gray order: 15 flips, each E += 2 s'_k F_k (s'_k the new value,
// F_k the field of spin k) and F_j += 2 s'_k J_jk for the other three.  Pass 1 keeps each
// thread's lowest (E, c); the S-th lowest of those 512 minima, real configurations, bounds the
// block's S-th lowest from above.  Pass 2 walks again and records every configuration at or
// below that bound (within the window W above it for float instances): never more than the
// block's 8192, one sort and the selection rule give the block list (its S lowest plus the
// float window).  The block lowers the global threshold; the lists then go through the
// pairwise merge rounds and the finalising kernels of k_select.cu.
#include <climits>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kSmallThreads = 512;
constexpr int kSmallWalkBits = 4;                     // spins walked by one thread

// Sort the first `count` records of the buffer (padded to a power of two) and return how many
// the keep rule retains: the first S, and for W > 0 every record within W of the S-th.
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

// one Gray step of a thread's walk over spins 0..3: step t flips spin k = ctz(t)
template <int t>
__device__ __forceinline__ void small_step(int& e, int (&F)[kSmallWalkBits], unsigned long long& c, const int* Jq,
                                           int n)
{
    constexpr int k = (t & 1) ? 0 : (t & 2) ? 1 : (t & 4) ? 2 : 3;
    const bool up = !((c >> k) & 1ull);            // new value of spin k is +1
    const unsigned fk = (unsigned)F[k];
    e = (int)((unsigned)e + (up ? fk << 1 : 0u - (fk << 1)));
#pragma unroll
    for (int j = 0; j < kSmallWalkBits; j++) {
        if (j == k) continue;
        const unsigned d = (unsigned)Jq[j * n + k] << 1;
        F[j] = (int)((unsigned)F[j] + (up ? d : 0u - d));
    }
    c ^= 1ull << k;
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_enum_kernel(const SmallParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);   // buf
    int* E = reinterpret_cast<int*>(C + p.buf);                             // buf
    int* Jq = E + p.buf;                                                    // n*n
    int* hq = Jq + p.n * p.n;                                               // n
    __shared__ int s_keep, s_EB, s_f[kSmallBlockBits];
    __shared__ unsigned s_count;
    const int n = p.n, S = p.S, cap = p.cap, tid = threadIdx.x, lane = tid & 31;
    const Prep* prep = p.prep;
    for (int i = tid; i < n * n; i += blockDim.x) Jq[i] = prep->Jq[i];
    for (int i = tid; i < n; i += blockDim.x) hq[i] = prep->hq[i];
    __syncthreads();
    const int W = prep->L.W;

    // the block's base configuration (its 13 low spins at -1): energy and the local fields of
    // those 13 spins, by the definition (Eq. (1))
    const unsigned long long cB = p.hiconst | ((unsigned long long)blockIdx.x << kSmallBlockBits);
    if (tid < 32) {
        int part = 0;
        for (int i = lane; i < n; i += 32) {
            int row = hq[i];
            for (int j = i + 1; j < n; j++) row += ((cB >> j) & 1ull) ? Jq[i * n + j] : -Jq[i * n + j];
            part += ((cB >> i) & 1ull) ? row : -row;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) s_EB = part;
    } else if (tid < 32 + kSmallBlockBits) {
        const int v = tid - 32;
        int f = hq[v];
        for (int j = 0; j < n; j++)
            if (j != v) f += ((cB >> j) & 1ull) ? Jq[v * n + j] : -Jq[v * n + j];
        s_f[v] = f;
    }
    __syncthreads();

    // this thread's start configuration: spins 4..12 set to the bits of tid (from -1 to +1, one
    // at a time: E += 2 f_v with f_v the current field), spins 0..3 at -1
    int e0 = s_EB;
    int F0[kSmallWalkBits];
#pragma unroll
    for (int k = 0; k < kSmallWalkBits; k++) F0[k] = s_f[k];
    for (int b = 0; b < kSmallBlockBits - kSmallWalkBits; b++) {
        if (!((tid >> b) & 1)) continue;
        const int v = kSmallWalkBits + b;
        unsigned fv = (unsigned)s_f[v];
        for (int b2 = 0; b2 < b; b2++)
            if ((tid >> b2) & 1) fv += (unsigned)Jq[v * n + kSmallWalkBits + b2] << 1;
        e0 = (int)((unsigned)e0 + (fv << 1));
#pragma unroll
        for (int k = 0; k < kSmallWalkBits; k++) F0[k] = (int)((unsigned)F0[k] + ((unsigned)Jq[k * n + v] << 1));
    }
    const unsigned long long c0 = cB | ((unsigned long long)tid << kSmallWalkBits);

    // pass 1: the lowest (E, c) of this thread's 16 configurations
    int e = e0, F[kSmallWalkBits];
    unsigned long long c = c0;
#pragma unroll
    for (int k = 0; k < kSmallWalkBits; k++) F[k] = F0[k];
    int mE = e;
    unsigned long long mC = c;
    auto track = [&]() { if (rec_less(e, c, mE, mC)) { mE = e; mC = c; } };
    small_step<1>(e, F, c, Jq, n); track();
    small_step<2>(e, F, c, Jq, n); track();
    small_step<3>(e, F, c, Jq, n); track();
    small_step<4>(e, F, c, Jq, n); track();
    small_step<5>(e, F, c, Jq, n); track();
    small_step<6>(e, F, c, Jq, n); track();
    small_step<7>(e, F, c, Jq, n); track();
    small_step<8>(e, F, c, Jq, n); track();
    small_step<9>(e, F, c, Jq, n); track();
    small_step<10>(e, F, c, Jq, n); track();
    small_step<11>(e, F, c, Jq, n); track();
    small_step<12>(e, F, c, Jq, n); track();
    small_step<13>(e, F, c, Jq, n); track();
    small_step<14>(e, F, c, Jq, n); track();
    small_step<15>(e, F, c, Jq, n); track();
    // the S-th lowest of the 512 thread minima (distinct configurations) bounds the block's S-th
    // lowest (E, c) from above
    E[tid] = mE;
    C[tid] = mC;
    __syncthreads();
    block_sort(E, C, kSmallThreads);
    const int kE = S <= kSmallThreads ? E[S - 1] : kEmptyE;
    const unsigned long long kC = S <= kSmallThreads ? C[S - 1] : kEmptyC;
    if (tid == 0) s_count = 0u;
    __syncthreads();

    // pass 2: record every configuration with (E, c) <= (kE, kC), or E <= kE + W for float
    // instances (the block's S lowest and its whole window); at most the block's 8192 fit the
    // buffer
    auto hit = [&]() {
        if (W == 0 ? rec_less(kE, kC, e, c) : (long long)e > (long long)kE + W) return;
        const unsigned slot = atomicAdd(&s_count, 1u);
        E[slot] = e;
        C[slot] = c;
    };
    e = e0;
    c = c0;
#pragma unroll
    for (int k = 0; k < kSmallWalkBits; k++) F[k] = F0[k];
    hit();
    small_step<1>(e, F, c, Jq, n); hit();
    small_step<2>(e, F, c, Jq, n); hit();
    small_step<3>(e, F, c, Jq, n); hit();
    small_step<4>(e, F, c, Jq, n); hit();
    small_step<5>(e, F, c, Jq, n); hit();
    small_step<6>(e, F, c, Jq, n); hit();
    small_step<7>(e, F, c, Jq, n); hit();
    small_step<8>(e, F, c, Jq, n); hit();
    small_step<9>(e, F, c, Jq, n); hit();
    small_step<10>(e, F, c, Jq, n); hit();
    small_step<11>(e, F, c, Jq, n); hit();
    small_step<12>(e, F, c, Jq, n); hit();
    small_step<13>(e, F, c, Jq, n); hit();
    small_step<14>(e, F, c, Jq, n); hit();
    small_step<15>(e, F, c, Jq, n); hit();
    __syncthreads();
    const int kept = sort_keep(E, C, (int)s_count, S, W, cap, p.hdr, &s_keep);

    for (int i = tid; i < cap; i += blockDim.x) {
        p.list_E[(size_t)blockIdx.x * cap + i] = i < kept ? E[i] : kEmptyE;
        p.list_C[(size_t)blockIdx.x * cap + i] = i < kept ? C[i] : kEmptyC;
    }
    if (tid == 0 && kept >= S) atomicMin(&p.hdr->tau, E[S - 1]);
}

}  // namespace

int small_lists(int free_bits) { return free_bits > kSmallBlockBits ? 1 << (free_bits - kSmallBlockBits) : 1; }

cudaError_t launch_small_enum(const SmallParams& p, cudaStream_t s)
{
    static_assert(kSmallThreads << kSmallWalkBits == 1 << kSmallBlockBits, "a block covers 2^13 configurations");
    if (p.free_bits < kSmallBlockBits || p.free_bits > kSmallMaxFreeBits || p.nlists != small_lists(p.free_bits) ||
        p.buf < (1 << kSmallBlockBits) || p.cap > p.buf)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)p.buf * 12 + (size_t)(p.n * p.n + p.n) * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(small_enum_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    small_enum_kernel<<<p.nlists, kSmallThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
