// Small search spaces (2^13 .. 2^20 configurations): the whole search in one launch.
//
// For spaces this small the walk of k_gray.cu has too little work to fill the GPU, and the
// launches around it (preparation, first threshold, merge rounds, finalisation) dominate the
// time of a call.  small_search_kernel, block b of G = 2^(free - 13):
//   1. fixed point, as the preparation kernel does it: emax = sum|J| + sum|h|, scale 2^q with
//      emax 2^q < 2^29, J_q, h_q by rounding, the rounding residual delta and the candidate
//      window W (every block computes the same values from the same inputs);
//   2. enumerates the 8192 configurations whose bits [13, free) equal b, exactly in int32.  The
//      block evaluates its base configuration (13 low spins at -1) and the fields of those
//      spins by the definition (Eq. (1)); thread t reaches its start (spins 4..12 = the bits of
//      t) by flipping those spins one at a time (E += 2 f_v, the current field of spin v), then
//      walks spins 0..3 in reflected Gray order: 15 flips, each E += 2 s'_k F_k (s'_k the new
//      value, F_k the field of spin k) and F_j += 2 s'_k J_jk for the other three.  Pass 1 keeps
//      each thread's lowest (E, c); the S-th lowest of those 512 minima, real configurations,
//      bounds the block's S-th lowest from above.  Pass 2 walks again and records every
//      configuration at or below that bound (within W above it for float instances): never
//      more than the block's 8192; one sort and the selection rule give the block list (its S
//      lowest plus the float window);
//   3. merges the lists pairwise up a binary tree without any wait: each tree node has a
//      ticket, and the second block to arrive at a node (both children written and fenced)
//      merges them (the running selection of Algorithm 1) and moves up;
//   4. the block that merges the root writes the status and the S results: E_q / 2^q for
//      integer instances; for float instances Eq. (1) evaluated exactly (the quantised energy
//      plus the rounding residuals, summed in 64-bit fixed point) and rounded once to FP64, then
//      a reselection by (E, c).
#include <cfloat>
#include <climits>
#include <cmath>
#include <utility>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kSmallThreads = 512;
constexpr int kSmallWalkBits = 4;                     // spins walked by one thread
constexpr int kSmallBuf = 1 << kSmallBlockBits;       // records of the block buffer: all 8192 fit
constexpr int kSmallResBits = 48;                     // fixed-point scale of the residuals: 2^(q+48)

__device__ __forceinline__ double load_value(const void* p, int dtype, size_t idx)
{
    if (dtype == 0) return (double)static_cast<const int*>(p)[idx];
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

__device__ double small_block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// thread 0: how many records of a sorted array the selection rule keeps (the first S, and for
// W > 0 every record within W of the S-th; beyond cap sets kErrWindow in *status)
__device__ int keep_rule(const int* E, int len, int S, int W, int cap, unsigned* status)
{
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
        *status |= kErrWindow;
    }
    return keep;
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

template <typename Visit, int... Ts>
__device__ __forceinline__ void small_walk(int& e, int (&F)[kSmallWalkBits], unsigned long long& c, const int* Jq,
                                           int n, Visit visit, std::integer_sequence<int, Ts...>)
{
    ((small_step<Ts + 1>(e, F, c, Jq, n), visit()), ...);
}

__global__ void __launch_bounds__(kSmallThreads, 1) small_search_kernel(const SmallParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);   // kSmallBuf
    // J and h in FP64; after quantisation the same words hold the residuals in fixed point
    double* Jd = reinterpret_cast<double*>(C + kSmallBuf);                  // n*n
    double* hd = Jd + p.n * p.n;                                            // n
    long long* Rq = reinterpret_cast<long long*>(Jd);                       // n*n (upper triangle)
    long long* Rh = reinterpret_cast<long long*>(hd);                       // n
    unsigned long long* key = reinterpret_cast<unsigned long long*>(hd + p.n);   // cap (root only)
    unsigned long long* cf = key + p.cap;                                   // cap (root only)
    double* red = reinterpret_cast<double*>(cf + p.cap);                    // kSmallThreads
    int* E = reinterpret_cast<int*>(red + kSmallThreads);                   // kSmallBuf
    int* Jq = E + kSmallBuf;                                                // n*n
    int* hq = Jq + p.n * p.n;                                               // n
    __shared__ int s_keep, s_EB, s_f[kSmallBlockBits], s_q, s_W;
    __shared__ unsigned s_count, s_status, s_ticket;
    const int n = p.n, S = p.S, cap = p.cap, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // 1. fixed point: the strict upper triangle of J and h, emax, q, J_q, h_q, delta, W
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        Jd[idx] = i < j ? load_value(p.J, p.dtype, idx) : 0.0;
    }
    for (int i = tid; i < n; i += blockDim.x) hd[i] = load_value(p.h, p.dtype, i);
    __syncthreads();
    double part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) part += fabs(Jd[idx]);
    for (int i = tid; i < n; i += blockDim.x) part += fabs(hd[i]);
    const double emax = small_block_sum(part, red);
    if (tid == 0) {
        unsigned status = 0u;
        int q = 0;
        if (emax > 0.0) {
            int ex;
            frexp(emax, &ex);                                 // emax < 2^ex
            q = kEmqLog2 - ex;
            if (p.dtype == 0) {
                if (q < 0) status |= kErrRange;               // integers beyond the int32 fixed point
                q = q > 16 ? 16 : (q < 0 ? 0 : q);
            } else {
                q = q > 200 ? 200 : (q < -200 ? -200 : q);
            }
        }
        if (!(emax < 1e300)) status |= kErrRange;             // inf / nan input
        if (p.range_flag && *p.range_flag) status |= kErrRange;   // found by the caller's own map
        s_q = q;
        s_status = status;
    }
    __syncthreads();
    const int q = s_q;
    // J_q, h_q by rounding; the residuals rho = x - x_q 2^-q (exact in FP64, |rho| <= 2^-(q+1))
    // are kept as integers round(rho 2^(q+48)) for the final re-evaluation, in place of x
    part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        if (i < j) {
            const double x = Jd[idx];
            const double r = rint(ldexp(x, q));
            Jq[idx] = Jq[j * n + i] = (int)r;
            const double rho = x - ldexp(r, -q);
            part += fabs(rho);
            Rq[idx] = __double2ll_rn(ldexp(rho, q + kSmallResBits));
        } else if (i == j) {
            Jq[idx] = 0;
        }
    }
    for (int i = tid; i < n; i += blockDim.x) {
        const double x = hd[i];
        const double r = rint(ldexp(x, q));
        hq[i] = (int)r;
        const double rho = x - ldexp(r, -q);
        part += fabs(rho);
        Rh[i] = __double2ll_rn(ldexp(rho, q + kSmallResBits));
    }
    const double delta = small_block_sum(part, red);
    if (tid == 0) {
        int W = 0;
        if (p.dtype != 0 && delta > 0.0) {
            // the quantisation (2 delta) and the FP64 evaluation error of the final reselection,
            // generously bounded, as in the preparation kernel
            const double eps = 8.0 * (double)n * (double)n * ldexp(1.0, -53) * emax;
            double w = ceil(ldexp(2.0 * delta + 2.0 * eps, q)) + 2.0;
            if (w > (double)(1 << 28)) { w = (double)(1 << 28); s_status |= kErrRange; }
            W = (int)w;
        }
        s_W = W;
    }
    __syncthreads();
    const int W = s_W;

    // 2a. the block's base configuration (13 low spins at -1): energy and the fields of those spins
    const unsigned long long cB = p.hiconst | ((unsigned long long)blockIdx.x << kSmallBlockBits);
    if (warp == 0) {
        int pe = 0;
        for (int i = lane; i < n; i += 32) {
            int row = hq[i];
            for (int j = i + 1; j < n; j++) row += ((cB >> j) & 1ull) ? Jq[i * n + j] : -Jq[i * n + j];
            pe += ((cB >> i) & 1ull) ? row : -row;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pe += __shfl_xor_sync(0xffffffffu, pe, o);
        if (lane == 0) s_EB = pe;
    } else if (tid < 32 + kSmallBlockBits) {
        const int v = tid - 32;
        int f = hq[v];
        for (int j = 0; j < n; j++)
            if (j != v) f += ((cB >> j) & 1ull) ? Jq[v * n + j] : -Jq[v * n + j];
        s_f[v] = f;
    }
    __syncthreads();

    // 2b. this thread's start: spins 4..12 set to the bits of tid, one at a time
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

    // 2c. pass 1: the lowest (E, c) of this thread's 16 configurations
    int e = e0, F[kSmallWalkBits];
    unsigned long long c = c0;
#pragma unroll
    for (int k = 0; k < kSmallWalkBits; k++) F[k] = F0[k];
    int mE = e;
    unsigned long long mC = c;
    small_walk(e, F, c, Jq, n, [&]() { if (rec_less(e, c, mE, mC)) { mE = e; mC = c; } },
               std::make_integer_sequence<int, 15>{});
    E[tid] = mE;
    C[tid] = mC;
    __syncthreads();
    block_sort(E, C, kSmallThreads);
    const int kE = S <= kSmallThreads ? E[S - 1] : kEmptyE;
    const unsigned long long kC = S <= kSmallThreads ? C[S - 1] : kEmptyC;
    __syncthreads();
    if (tid == 0) s_count = 0u;
    __syncthreads();

    // 2d. pass 2: every configuration with (E, c) <= (kE, kC), or E <= kE + W for float instances
    auto record = [&]() {
        if (W == 0 ? rec_less(kE, kC, e, c) : (long long)e > (long long)kE + W) return;
        const unsigned slot = atomicAdd(&s_count, 1u);
        E[slot] = e;
        C[slot] = c;
    };
    e = e0;
    c = c0;
#pragma unroll
    for (int k = 0; k < kSmallWalkBits; k++) F[k] = F0[k];
    record();
    small_walk(e, F, c, Jq, n, record, std::make_integer_sequence<int, 15>{});
    __syncthreads();
    const int count = (int)s_count;
    int len = 64;
    while (len < count) len <<= 1;
    for (int i = count + tid; i < len; i += blockDim.x) {
        E[i] = kEmptyE;
        C[i] = kEmptyC;
    }
    block_sort(E, C, len);
    if (tid == 0) s_keep = keep_rule(E, len, S, W, cap, &s_status);
    __syncthreads();
    int kept = s_keep;

    // 3. up the merge tree: node (level, i) is stored at leaf slot i 2^level
    const int G = (int)gridDim.x;
    int node = blockIdx.x, level = 0, toff = 0;
    while ((G >> level) > 1) {
        const size_t slot = (size_t)node << level;
        for (int i = tid; i < cap; i += blockDim.x) {
            if (i >= kept) {
                E[i] = kEmptyE;
                C[i] = kEmptyC;
            }
            p.list_E[slot * cap + i] = E[i];
            p.list_C[slot * cap + i] = C[i];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (s_status) atomicOr(&p.aux[0], s_status);     // conditions found so far travel to the root
            __threadfence();
            s_ticket = atomicAdd(&p.aux[1 + toff + (node >> 1)], 1u);
            __threadfence();
        }
        __syncthreads();
        if (s_ticket == 0u) return;                          // the sibling merges this node
        // both children written: this block's own list is still in [0, cap); the sibling's goes
        // into [cap, 2 cap)
        const size_t sib = (size_t)(node ^ 1) << level;
        for (int i = tid; i < cap; i += blockDim.x) {
            E[cap + i] = *(volatile const int*)&p.list_E[sib * cap + i];
            C[cap + i] = *(volatile const unsigned long long*)&p.list_C[sib * cap + i];
        }
        block_merge_halves(E, C, 2 * cap);
        if (tid == 0) s_keep = keep_rule(E, 2 * cap, S, W, cap, &s_status);
        __syncthreads();
        kept = s_keep;
        toff += G >> (level + 1);
        node >>= 1;
        level++;
    }

    // 4. the root: the status word, then the S results
    if (tid == 0) {
        p.hdr->status = s_status | atomicOr(&p.aux[0], 0u);
        p.hdr->tau = kept >= S ? E[S - 1] : INT_MAX;        // the S-th lowest quantised energy
        p.hdr->task_next = 0ull;
        p.hdr->spill_count = 0u;
    }
    if (p.dtype == 0) {
        // integer instances: E_q = E 2^q exactly
        for (int k = tid; k < S; k += blockDim.x) {
            static_cast<long long*>(p.energies)[k] = (long long)((k < kept ? E[k] : kEmptyE) >> q);
            p.states[k] = k < kept ? C[k] : kEmptyC;
        }
        return;
    }
    // float instances: every kept record re-evaluated, one thread per record.  Eq. (1) splits
    // into the quantised energy and the residual terms, E(c) = 2^-q (E_q(c) + R(c)), with
    // R(c) = sum_{i<j} rho_ij s_i s_j + sum_i rho_i s_i summed exactly in 64-bit fixed point
    // (scale 2^(q+48): every term |rho'| <= 2^47, at most 2144 terms), then one rounding to FP64.
    // The truncation of the residuals to that scale, at most 2^-(q+37) in all, lies far below
    // the FP64 unit of E (2^-q ~ emax 2^-29).  Integer arithmetic instead of an FP64 sum: the
    // FP64 unit of this GPU issues 2 lanes per clock per SM.  Then the exact reselection by
    // (E, c), with E mapped to an order-preserving unsigned key.
    int flen = 2;
    while (flen < kept || flen < S) flen <<= 1;           // <= cap: S <= cap / 2
    for (int r = tid; r < flen; r += blockDim.x) {
        if (r >= kept) {
            key[r] = ~0ull;
            cf[r] = kEmptyC;
            continue;
        }
        const unsigned long long cc = C[r];
        long long R = 0;
        for (int i = 0; i < n; i++) {
            long long row = Rh[i];
            const long long* Ri = Rq + i * n;
            for (int j = i + 1; j < n; j++) row += ((cc >> j) & 1ull) ? Ri[j] : -Ri[j];
            R += ((cc >> i) & 1ull) ? row : -row;
        }
        const double e = ldexp((double)E[r], -q) + ldexp((double)R, -q - kSmallResBits);
        const unsigned long long u = (unsigned long long)__double_as_longlong(e);
        key[r] = (u >> 63) ? ~u : u | 0x8000000000000000ull;
        cf[r] = cc;
    }
    __syncthreads();
    block_sort(key, cf, flen);
    for (int k = tid; k < S; k += blockDim.x) {
        const unsigned long long u = key[k];
        static_cast<double*>(p.energies)[k] =
            u == ~0ull ? DBL_MAX : __longlong_as_double((long long)((u >> 63) ? u & 0x7fffffffffffffffull : ~u));
        p.states[k] = cf[k];
    }
}

}  // namespace

int small_lists(int free_bits) { return free_bits > kSmallBlockBits ? 1 << (free_bits - kSmallBlockBits) : 1; }

size_t small_smem_bytes(int n, int cap)
{
    return (size_t)kSmallBuf * 12 + (size_t)(n * n + n) * 12 + (size_t)cap * 16 + (size_t)kSmallThreads * 8;
}

cudaError_t launch_small(const SmallParams& p, cudaStream_t s)
{
    static_assert(kSmallThreads << kSmallWalkBits == 1 << kSmallBlockBits, "a block covers 2^13 configurations");
    if (p.free_bits < kSmallBlockBits || p.free_bits > kSmallMaxFreeBits || p.nlists != small_lists(p.free_bits) ||
        2 * p.cap > kSmallBuf || p.S > p.cap)
        return cudaErrorInvalidValue;
    // the status accumulator and the merge tree's tickets (nlists - 1) start at zero
    cudaError_t e = cudaMemsetAsync(p.aux, 0, (size_t)p.nlists * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const size_t smem = small_smem_bytes(p.n, p.cap);
    e = ensure_smem(reinterpret_cast<const void*>(small_search_kernel), smem);
    if (e != cudaSuccess) return e;
    small_search_kernel<<<p.nlists, kSmallThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
