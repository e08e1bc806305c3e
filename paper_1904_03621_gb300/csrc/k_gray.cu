// Gray-code enumeration of all configurations with threshold-pruned top-S
// capture (steps A1 and A3).
//
// The paper evaluates each configuration independently in O(n^2) (one
// state per thread, Sec. 4.2) and selects the lowest S per chunk
// (Algorithm 1, Sec. 3).  Here each walk owns a fixed prefix of high spins
// (a "task") and visits the remaining spins in reflected Gray-code order, so
// consecutive configurations differ by one spin and the energy changes by
// dE = 2 s_new F_k (F_k the local field on the flipped spin k).
//
// Bit layout of a configuration c (bit i = spin i, 1 = +1):
//   [0, B)         inner spins: walked by a fully unrolled (2^B - 1)-step block,
//                  B = 10 for searches of >= 2^42 configurations, else 9
//   [B, B+m)       middle spins: walked one flip per block (dynamic index)
//   [B+m, free)    task index (prefix) of the walk
//   [free, n)      fixed bits (subspace mode, Sec. 3, Eq. (6))
//
// Arithmetic: the quantised instance is exact in int32.  Per walk we keep
// E0 (energy with all inner spins at -1), G_k = 2 F_k for the B inner spins
// (fields from non-inner spins) and the local fields of 4 middle spins.
// Inside a block, E(g) = E0 + sum_{k in g} G_k + T[g] - T[0].  The unrolled
// walk runs on 16-bit values floor((E + 2^31) / 2^16), two walks packed per
// 32-bit register: one IADD3 advances two walks by one flip and one 16x2
// minimum folds them into a running minimum.  A block whose 16-bit minimum
// reaches the threshold is rescanned exactly in int32, and only exact hits
// are recorded.  Error bound of the 16-bit value x(g) of a configuration:
//   E(g)/2^16 - (B + 2) < x(g) - 2^15 <= E(g)/2^16 + 1,
// so x(g) <= floor((tau + 2^31) / 2^16) + 1 catches every E(g) <= tau.
//
// Selection: hits go to a shared-memory buffer (spill area in the
// workspace when full).  At segment boundaries the block merges the buffer
// into its sorted list of the lowest records, tightens its threshold and
// publishes it with atomicMin; blocks read the global threshold back.
#include <climits>
#include <utility>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

__host__ __device__ constexpr int cx_ctz(int t) { return (t & 1) ? 0 : 1 + cx_ctz(t >> 1); }
// value (1 = +1) of the spin flipped by step t of the reflected Gray code
__host__ __device__ constexpr bool cx_up(int t) { return (((t ^ (t >> 1)) >> cx_ctz(t)) & 1) != 0; }

template <int IB>
struct Packed {
    unsigned Xa, Xb, M;
    unsigned Ga[IB], Gb[IB];
};

template <int IB, int t>
__device__ __forceinline__ void inner_step(Packed<IB>& w, const GrayParams& p)
{
    constexpr int k = cx_ctz(t);
    constexpr bool up = cx_up(t);
    w.Xa += (up ? w.Ga[k] : 0u - w.Ga[k]) + p.dT16[t];
    w.Xb += (up ? w.Gb[k] : 0u - w.Gb[k]) + p.dT16[t];
    w.M = __vminu2(__vminu2(w.M, w.Xa), w.Xb);
}

template <int IB, int... Ts>
__device__ __forceinline__ void inner_walk(Packed<IB>& w, const GrayParams& p, std::integer_sequence<int, Ts...>)
{
    (inner_step<IB, Ts + 1>(w, p), ...);
}

// integer packing hi * 2^16 + lo of the 16-bit views (floor(x / 2^16)) of two int32 values
__device__ __forceinline__ unsigned pack_hi16(int lo, int hi)
{
    return ((unsigned)(hi >> 16) << 16) + (unsigned)(lo >> 16);
}

__device__ __forceinline__ unsigned pack_energy(int lo, int hi)
{
    return (((unsigned)hi + 0x80000000u) & 0xffff0000u) | (((unsigned)lo + 0x80000000u) >> 16);
}

struct Smem {
    int* Jq;                 // n*n
    int* hq;                 // kMaxN
    int* T;                  // 256
    int (*col)[16];          // kMaxN x 16
    int* E;                  // 2 * cap
    unsigned long long* C;   // 2 * cap
};

__device__ __forceinline__ void record(const GrayParams& p, const Smem& s, unsigned* buf_count, int e,
                                       unsigned long long c)
{
    unsigned slot = atomicAdd(buf_count, 1u);
    if (slot < (unsigned)p.list_cap) {
        s.E[p.list_cap + slot] = e;
        s.C[p.list_cap + slot] = c;
        return;
    }
    unsigned g = atomicAdd(&p.hdr->spill_count, 1u);
    if (g < p.spill_cap) {
        p.spill_E[g] = e;
        p.spill_C[g] = c;
    } else {
        atomicOr(&p.hdr->status, kErrSpill);
    }
}

// local field on spin j (inner spins at -1 are part of cfg) of one configuration
__device__ __forceinline__ int field_at(const Smem& s, int n, int j, unsigned long long cfg)
{
    int f = s.hq[j];
    const int* row = s.Jq + j * n;
    for (int i = 0; i < n; i++) {
        int v = row[i];
        f += ((cfg >> i) & 1ull) ? v : -v;
    }
    return f;
}

}  // namespace

template <int IB>
__global__ void __launch_bounds__(kGrayThreads, 2) gray_kernel(const __grid_constant__ GrayParams p)
{
    constexpr int IS = 1 << IB;                  // configurations per unrolled block and walk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = p.n;
    const int cap = p.list_cap;
    Smem s;
    s.C = reinterpret_cast<unsigned long long*>(smem_raw);                  // 2*cap
    s.E = reinterpret_cast<int*>(s.C + 2 * cap);                            // 2*cap
    s.col = reinterpret_cast<int(*)[16]>(s.E + 2 * cap);                    // kMaxN*16
    s.T = reinterpret_cast<int*>(s.col + kMaxN);                            // 256
    s.hq = s.T + kGrayMaxInnerSteps;                                               // kMaxN
    s.Jq = s.hq + kMaxN;                                                    // n*n

    __shared__ unsigned s_buf_count;
    __shared__ int s_list_count, s_kE;               // s_kE, s_kC: S-th record of the block list
    __shared__ unsigned long long s_batch, s_kC;

    const int tid = threadIdx.x;
    const Prep* prep = p.prep;
    for (int i = tid; i < n * n; i += blockDim.x) s.Jq[i] = prep->Jq[i];
    for (int i = tid; i < kMaxN; i += blockDim.x) s.hq[i] = prep->hq[i];
    for (int i = tid; i < IS; i += blockDim.x) s.T[i] = prep->T[i];
    for (int i = tid; i < kMaxN * 16; i += blockDim.x) s.col[i / 16][i % 16] = prep->colJ[i / 16][i % 16];
    if (tid == 0) {
        s_buf_count = 0u;
        s_list_count = 0;
        s_kE = kEmptyE;
        s_kC = kEmptyC;
    }
    __syncthreads();

    const int S = p.S, W = p.W, m = p.m;
    const int walk_shift = IB + m;       // task index sits above inner + middle spins
    const unsigned nblocks = 1u << m;
    const unsigned seg_mask = (1u << p.seg_log2) - 1u;

    // screening threshold in quantised units and its 16-bit view; for
    // integer instances (W = 0) records at the block's S-th energy are kept
    // only below the block's S-th configuration (key order (E, c))
    int tau_scr = 0, tie_E = kEmptyE;
    unsigned long long tie_C = kEmptyC;
    unsigned thr16 = 0;
    auto refresh_threshold = [&]() {
        int tg = *(volatile int*)&p.hdr->tau;
        int t = min(s_kE, tg);
        tie_E = (W == 0) ? s_kE : kEmptyE;
        tie_C = s_kC;
        long long ts = (long long)t + W;
        if (ts > (1ll << 30)) ts = 1ll << 30;
        tau_scr = (int)ts;
        unsigned th = (((unsigned)tau_scr + 0x80000000u) >> 16) + 1u;
        thr16 = th > 0xffffu ? 0xffffu : th;
    };
    refresh_threshold();

    for (;;) {
        if (tid == 0) s_batch = atomicAdd(&p.hdr->task_next, (unsigned long long)(kGrayThreads * kWalks));
        __syncthreads();
        const unsigned long long base = s_batch;
        __syncthreads();
        if (base >= p.ntasks) break;

        // ---- per-walk state at the start of the task (middle and inner spins all -1)
        int E0[kWalks], G[kWalks][IB], Fm[kWalks][kKeep];
        unsigned long long cfg0[kWalks];
        bool active[kWalks];
#pragma unroll
        for (int w = 0; w < kWalks; w++) {
            unsigned long long task = base + (unsigned long long)(tid * kWalks + w);
            active[w] = task < p.ntasks;
            if (!active[w]) task = 0;   // a valid walk whose hits are ignored
            cfg0[w] = p.hiconst | (task << walk_shift);
        }
#pragma unroll
        for (int w = 0; w < kWalks; w++) {
            const unsigned long long c = cfg0[w];
            int e = 0;
            for (int i = 0; i < n; i++) {
                int row = s.hq[i];
                const int* Ji = s.Jq + i * n;
                for (int j = i + 1; j < n; j++) {
                    int v = Ji[j];
                    row += ((c >> j) & 1ull) ? v : -v;
                }
                e += ((c >> i) & 1ull) ? row : -row;
            }
            E0[w] = e;
#pragma unroll
            for (int k = 0; k < IB; k++) {
                int f = s.hq[k];
                const int* Jk = s.Jq + k * n;
                for (int j = IB; j < n; j++) {
                    int v = Jk[j];
                    f += ((c >> j) & 1ull) ? v : -v;
                }
                G[w][k] = 2 * f;
            }
#pragma unroll
            for (int r = 0; r < kKeep; r++) Fm[w][r] = field_at(s, n, IB + r, c);
        }

        Packed<IB> pk;
#pragma unroll
        for (int k = 0; k < IB; k++) {
            pk.Ga[k] = pack_hi16(G[0][k], G[1][k]);
            pk.Gb[k] = pack_hi16(G[2][k], G[3][k]);
        }

        unsigned long long cmid = 0ull;   // middle spins of the current block: gray(u) << 8
        for (unsigned u = 0; u < nblocks; ++u) {
            // ---- one block: 512 configurations per walk, four walks
            pk.Xa = pack_energy(E0[0], E0[1]);
            pk.Xb = pack_energy(E0[2], E0[3]);
            pk.M = __vminu2(pk.Xa, pk.Xb);
            inner_walk<IB>(pk, p, std::make_integer_sequence<int, IS - 1>{});
            const bool flag_lo = (pk.M & 0xffffu) <= thr16;
            const bool flag_hi = (pk.M >> 16) <= thr16;
            if (flag_lo || flag_hi) {
#pragma unroll
                for (int w = 0; w < kWalks; w++) {
                    const bool lane_hi = (w & 1) != 0;
                    if (!active[w] || !(lane_hi ? flag_hi : flag_lo)) continue;
                    const unsigned ebase = (unsigned)E0[w] - (unsigned)s.T[0];
                    const unsigned long long cb = cfg0[w] | cmid;
                    for (int t = 0; t < IS; t++) {
                        const int g = t ^ (t >> 1);
                        unsigned acc = ebase + (unsigned)s.T[g];
#pragma unroll
                        for (int k = 0; k < IB; k++) acc += ((g >> k) & 1) ? (unsigned)G[w][k] : 0u;
                        const int e = (int)acc;   // E(g) = E0 + sum_{k in g} G_k + T[g] - T[0]
                        const unsigned long long c = cb | (unsigned long long)g;
                        if (e <= tau_scr && !(e == tie_E && c > tie_C)) record(p, s, &s_buf_count, e, c);
                    }
                }
            }

            // ---- segment boundary (dense at the start of a task): merge the buffer into the block list
            if ((u & seg_mask) == seg_mask || u < 16u || u + 1 == nblocks) {
                __syncthreads();
                const unsigned bc = s_buf_count;
                __syncthreads();
                if (bc > 0u) {
                    const int lc = s_list_count;
                    const int nb = bc < (unsigned)cap ? (int)bc : cap;
                    for (int i = tid; i < 2 * cap; i += blockDim.x) {
                        if ((i >= lc && i < cap) || i >= cap + nb) {
                            s.E[i] = kEmptyE;
                            s.C[i] = kEmptyC;
                        }
                    }
                    block_sort(s.E, s.C, 2 * cap);
                    if (tid == 0) {
                        const int total = lc + nb;
                        int keep = total;
                        if (total >= S) {
                            const int K = s.E[S - 1];
                            keep = S;
                            if (W > 0) {
                                long long lim = (long long)K + W;
                                keep = upper_bound_key(s.E, 2 * cap, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
                                if (keep > total) keep = total;
                                if (keep > cap) { keep = cap; atomicOr(&p.hdr->status, kErrWindow); }
                            }
                            s_kE = K;
                            s_kC = s.C[S - 1];
                            atomicMin(&p.hdr->tau, K);
                        } else if (keep > cap) {
                            keep = cap;   // cannot happen: S <= cap / 2
                        }
                        s_list_count = keep;
                        s_buf_count = 0u;
                    }
                    __syncthreads();
                }
                refresh_threshold();
            }

            // ---- flip one middle spin: j = IB + ctz(u + 1)
            if (u + 1 < nblocks) {
                const unsigned u1 = u + 1;
                const int jrel = __ffs(u1) - 1;
                const int j = IB + jrel;
                const bool up = ((u1 ^ (u1 >> 1)) >> jrel) & 1u;
                int F[kWalks];
                if (jrel < kKeep) {
#pragma unroll
                    for (int w = 0; w < kWalks; w++) {
                        int f = Fm[w][0];
#pragma unroll
                        for (int r = 1; r < kKeep; r++) f = (jrel == r) ? Fm[w][r] : f;
                        F[w] = f;
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < kWalks; w++) F[w] = field_at(s, n, j, cfg0[w] | cmid);
                }
                static_assert(IB + kKeep <= 16, "column table holds 16 entries");
                int colv[16];
#pragma unroll
                for (int q4 = 0; q4 < 4; q4++) {
                    const int4 cv = *reinterpret_cast<const int4*>(&s.col[j][4 * q4]);
                    colv[4 * q4 + 0] = cv.x;
                    colv[4 * q4 + 1] = cv.y;
                    colv[4 * q4 + 2] = cv.z;
                    colv[4 * q4 + 3] = cv.w;
                }
                // unsigned arithmetic: exact modulo 2^32, and every true result fits in int32
#pragma unroll
                for (int w = 0; w < kWalks; w++) {
                    const unsigned dE = (unsigned)F[w] << 1;
                    E0[w] = (int)((unsigned)E0[w] + (up ? dE : 0u - dE));
#pragma unroll
                    for (int k = 0; k < IB; k++) {
                        const unsigned d = (unsigned)colv[k] << 2;
                        G[w][k] = (int)((unsigned)G[w][k] + (up ? d : 0u - d));
                    }
#pragma unroll
                    for (int r = 0; r < kKeep; r++) {
                        const unsigned d = (unsigned)colv[IB + r] << 1;
                        Fm[w][r] = (int)((unsigned)Fm[w][r] + (up ? d : 0u - d));
                    }
                }
                cmid ^= 1ull << j;
#pragma unroll
                for (int k = 0; k < IB; k++) {
                    pk.Ga[k] = pack_hi16(G[0][k], G[1][k]);
                    pk.Gb[k] = pack_hi16(G[2][k], G[3][k]);
                }
            }
        }
    }

    // ---- write the block list (sorted, empty slots padded)
    const int lc = s_list_count;
    for (int i = tid; i < cap; i += blockDim.x) {
        p.list_E[(size_t)blockIdx.x * cap + i] = i < lc ? s.E[i] : kEmptyE;
        p.list_C[(size_t)blockIdx.x * cap + i] = i < lc ? s.C[i] : kEmptyC;
    }
}

size_t gray_smem_bytes(int n, int list_cap)
{
    return (size_t)2 * list_cap * 8 + (size_t)2 * list_cap * 4 + kMaxN * 16 * 4 + kGrayMaxInnerSteps * 4 +
           kMaxN * 4 + (size_t)n * n * 4;
}

// both block sizes use the same shared memory and at most 128 registers (2 blocks per SM)
int gray_blocks_per_sm(int list_cap)
{
    int blocks = 0;
    size_t smem = gray_smem_bytes(kMaxN, list_cap);
    if (cudaFuncSetAttribute(gray_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, gray_kernel<10>, kGrayThreads, smem) != cudaSuccess)
        return 0;
    return blocks;
}

template <int IB>
cudaError_t launch_gray_ib(const GrayParams& p, int grid, cudaStream_t s)
{
    size_t smem = gray_smem_bytes(p.n, p.list_cap);
    cudaError_t e = cudaFuncSetAttribute(gray_kernel<IB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gray_smem_bytes(kMaxN, p.list_cap));
    if (e != cudaSuccess) return e;
    gray_kernel<IB><<<grid, kGrayThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gray(const GrayParams& p, int grid, cudaStream_t s)
{
    return p.inner_bits == 10 ? launch_gray_ib<10>(p, grid, s) : launch_gray_ib<9>(p, grid, s);
}

}  // namespace bf
