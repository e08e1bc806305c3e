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
// (fields from non-inner spins) and the local fields of 4 middle spins.  A
// block takes kGrayThreads * kWalks consecutive tasks at a time.
// Inside a block, E(g) = E0 + sum_{k in g} G_k + T[g] - T[0].  The unrolled
// walk runs on 16-bit values floor((E + 2^31) / 2^16), two walks packed per
// 32-bit register: one IADD3 advances two walks by one flip and one 16x2
// minimum folds them into a running minimum.  A block whose 16-bit minimum
// reaches the threshold is rescanned exactly in int32, and only exact hits
// are recorded.  Error bound of the 16-bit value x(g) of a configuration:
//   E(g)/2^16 - (B + 2) < x(g) - 2^15 <= E(g)/2^16 + 1,
// so x(g) <= floor((tau + 2^31) / 2^16) + 1 catches every E(g) <= tau.  The
// warp rescans its flagged walks together, 2^B / 32 configurations per lane.
//
// Selection: hits go to a shared-memory buffer (spill area in the
// workspace when full).  At segment boundaries the block merges the buffer
// into its sorted list of the lowest records, tightens its threshold and
// publishes it with atomicMin; blocks read the global threshold back.
#include <climits>
#include <cstddef>
#include <mutex>
#include <utility>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kVarBits = 10;   // task-index bits that differ within one batch of tasks
static_assert(kGrayThreads * kWalks == 1 << kVarBits, "a batch is 2^kVarBits tasks");

// packed 16-bit pair-energy increments of the unrolled steps (Prep::L.dT16 of the search being
// run), copied in by launch_gray; read as constant-bank operands of the step additions
__constant__ unsigned c_dT16[kGrayMaxInnerSteps];

__host__ __device__ constexpr int cx_ctz(int t) { return (t & 1) ? 0 : 1 + cx_ctz(t >> 1); }
// value (1 = +1) of the spin flipped by step t of the reflected Gray code
__host__ __device__ constexpr bool cx_up(int t) { return (((t ^ (t >> 1)) >> cx_ctz(t)) & 1) != 0; }

template <int IB>
struct Packed {
    unsigned Xa, Xb, M;
    unsigned Ga[IB], Gb[IB];
};

template <int IB, int t>
__device__ __forceinline__ void inner_step(Packed<IB>& w)
{
    constexpr int k = cx_ctz(t);
    constexpr bool up = cx_up(t);
    w.Xa += (up ? w.Ga[k] : 0u - w.Ga[k]) + c_dT16[t];
    w.Xb += (up ? w.Gb[k] : 0u - w.Gb[k]) + c_dT16[t];
    w.M = __vminu2(__vminu2(w.M, w.Xa), w.Xb);
}

template <int IB, int... Ts>
__device__ __forceinline__ void inner_walk(Packed<IB>& w, std::integer_sequence<int, Ts...>)
{
    (inner_step<IB, Ts + 1>(w), ...);
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
    int* T;                  // 2^B
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

// Exact rescan of one walk's block by a whole warp.  Lane L takes the R = 2^B / 32
// Gray steps t = L*R .. L*R + R - 1: it sums the fields of its first configuration
// g(t) = t ^ (t >> 1), then follows one flip per step (step t flips bit ctz(t)).
// E(g) = ebase + T[g] + sum_{k in g} G_k, with ebase = E0 - T[0]; G is the walk's
// field row, staged in shared memory by the lane that owns the walk.
template <int IB>
__device__ __forceinline__ void warp_rescan(const GrayParams& p, const Smem& s, unsigned* buf_count, unsigned ebase,
                                            const int* G, unsigned long long cb, int tau, int tie_E,
                                            unsigned long long tie_C, int lane)
{
    constexpr unsigned R = (1u << IB) / 32u;
    unsigned t = (unsigned)lane * R;
    unsigned g = t ^ (t >> 1);
    unsigned sg = 0u;
#pragma unroll
    for (int k = 0; k < IB; k++) sg += ((g >> k) & 1u) ? (unsigned)G[k] : 0u;
    for (unsigned i = 0; i < R; i++) {
        if (i > 0) {
            const int k = __ffs(++t) - 1;
            g ^= 1u << k;
            sg += ((g >> k) & 1u) ? (unsigned)G[k] : 0u - (unsigned)G[k];
        }
        const int e = (int)(ebase + (unsigned)s.T[g] + sg);
        const unsigned long long c = cb | g;
        if (e <= tau && !(e == tie_E && c > tie_C)) record(p, s, buf_count, e, c);
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
    s.T = reinterpret_cast<int*>(s.col + kMaxN);                            // 2^B
    s.hq = s.T + kGrayMaxInnerSteps;                                               // kMaxN
    s.Jq = s.hq + kMaxN;                                                    // n*n

    __shared__ unsigned s_buf_count;
    __shared__ int s_list_count, s_kE;               // s_kE, s_kC: S-th record of the block list
    __shared__ unsigned long long s_batch, s_kC;
    __shared__ int s_ER[2], s_fR[kVarBits], s_gR[IB], s_fmR[kKeep];   // energy and fields of cR
    __shared__ int s_Gw[kGrayThreads / 32][IB];                         // field row of a walk being rescanned

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const Prep* prep = p.prep;
    if (*(volatile unsigned*)&p.hdr->status & kErrRange) {
        // the instance is outside the fixed-point range (reported by the workspace status): no walk
        for (int i = tid; i < cap; i += blockDim.x) {
            p.list_E[(size_t)blockIdx.x * cap + i] = kEmptyE;
            p.list_C[(size_t)blockIdx.x * cap + i] = kEmptyC;
        }
        return;
    }
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

    const int S = p.S, W = prep->L.W, m = p.m;
    // zero-field instances (prep->L.z2): the lower half of the task range, whose top task bit
    // (spin n - 1) is 0; the final selection adds the mirrors
    const unsigned long long ntasks = p.ntasks >> prep->L.z2;
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
        if (base >= ntasks) break;

        // ---- per-walk state at the start of the task (middle and inner spins all -1)
        int E0[kWalks], G[kWalks][IB], Fm[kWalks][kKeep];
        unsigned long long cfg0[kWalks];
        bool active[kWalks];
        if constexpr (IB < kGrayMaxInnerBits) {
            // Short tasks (the 9-spin block serves searches below 2^42 configurations, whose
            // tasks hold few blocks): the setup is shared by the block.
            // The batch's kGrayThreads * kWalks tasks share every spin except the nv lowest
            // task-index bits, which walk x = tid * kWalks + w sets to x.  The block first
            // evaluates cR, the batch's configuration with those nv spins at -1: its energy
            // and the local fields the walks start from.  Each walk then adds the flips of its
            // own bits (Eq. (1)): flipping spin v from -1 to +1 adds 2 f_v to E and 2 J_jv to
            // the field on spin j, and each pair of flipped spins adds 4 J_vv' to E.
            const int nv = p.nh < kVarBits ? p.nh : kVarBits;
            const unsigned long long cR = p.hiconst | (base << walk_shift);
            {
                int part = 0;
                if (tid < kMaxN) {
                    const int i = tid;
                    if (i < n) {
                        int row = s.hq[i];
                        const int* Ji = s.Jq + i * n;
                        for (int j = i + 1; j < n; j++) {
                            const int v = Ji[j];
                            row += ((cR >> j) & 1ull) ? v : -v;
                        }
                        part = ((cR >> i) & 1ull) ? row : -row;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    if ((tid & 31) == 0) s_ER[tid >> 5] = part;
                } else if (tid < kMaxN + kVarBits) {
                    const int b = tid - kMaxN;
                    if (b < nv) s_fR[b] = field_at(s, n, walk_shift + b, cR);
                } else if (tid < kMaxN + kVarBits + IB) {
                    const int k = tid - kMaxN - kVarBits;
                    int f = s.hq[k];
                    const int* Jk = s.Jq + k * n;
                    for (int j = IB; j < n; j++) {
                        const int v = Jk[j];
                        f += ((cR >> j) & 1ull) ? v : -v;
                    }
                    s_gR[k] = f;
                } else if (tid < kMaxN + kVarBits + IB + kKeep) {
                    const int r = tid - kMaxN - kVarBits - IB;
                    s_fmR[r] = field_at(s, n, IB + r, cR);
                }
            }
            __syncthreads();

            // flips of the task bits 2..nv-1 that the thread's walks share (unsigned
            // arithmetic: exact modulo 2^32, and every true result fits in int32)
            const unsigned xt = (unsigned)tid * kWalks;
            const unsigned vmask = (1u << nv) - 1u;
            unsigned Et = 0u, P0 = 0u, P1 = 0u;
            unsigned Gt[IB], Ft[kKeep];
#pragma unroll
            for (int k = 0; k < IB; k++) Gt[k] = 0u;
#pragma unroll
            for (int r = 0; r < kKeep; r++) Ft[r] = 0u;
            for (int b = 2; b < nv; b++) {
                const unsigned on = 0u - ((xt >> b) & 1u);
                const int v = walk_shift + b;
                const int* Jv = s.Jq + v * n + walk_shift;
                unsigned pair = 0u;
                for (int b2 = 2; b2 < b; b2++) pair += (unsigned)Jv[b2] & (0u - ((xt >> b2) & 1u));
                Et += ((unsigned)s_fR[b] * 2u + pair * 4u) & on;
                P0 += (unsigned)Jv[0] & on;
                P1 += (unsigned)Jv[1] & on;
                int colv[16];
#pragma unroll
                for (int q4 = 0; q4 < 4; q4++) {
                    const int4 cv = *reinterpret_cast<const int4*>(&s.col[v][4 * q4]);
                    colv[4 * q4 + 0] = cv.x;
                    colv[4 * q4 + 1] = cv.y;
                    colv[4 * q4 + 2] = cv.z;
                    colv[4 * q4 + 3] = cv.w;
                }
#pragma unroll
                for (int k = 0; k < IB; k++) Gt[k] += ((unsigned)colv[k] * 4u) & on;
#pragma unroll
                for (int r = 0; r < kKeep; r++) Ft[r] += ((unsigned)colv[IB + r] * 2u) & on;
            }
            const unsigned ER = (unsigned)s_ER[0] + (unsigned)s_ER[1];

#pragma unroll
            for (int w = 0; w < kWalks; w++) {
                // an inactive walk (task >= ntasks) keeps a valid configuration; its hits are ignored
                active[w] = base + (unsigned long long)(xt + w) < ntasks;
                unsigned e = ER + Et;
                unsigned g[IB], fm[kKeep];
#pragma unroll
                for (int k = 0; k < IB; k++) g[k] = (unsigned)s_gR[k] * 2u + Gt[k];
#pragma unroll
                for (int r = 0; r < kKeep; r++) fm[r] = (unsigned)s_fmR[r] + Ft[r];
                unsigned long long c = cR | ((unsigned long long)(xt & vmask) << walk_shift);
#pragma unroll
                for (int b = 0; b < 2; b++) {
                    if (!((w >> b) & 1) || b >= nv) continue;
                    const int v = walk_shift + b;
                    unsigned d = (unsigned)s_fR[b] * 2u + (b == 0 ? P0 : P1) * 4u;
                    if (b == 1 && (w & 1)) d += (unsigned)s.Jq[v * n + walk_shift] * 4u;
                    e += d;
#pragma unroll
                    for (int k = 0; k < IB; k++) g[k] += (unsigned)s.col[v][k] * 4u;
#pragma unroll
                    for (int r = 0; r < kKeep; r++) fm[r] += (unsigned)s.col[v][IB + r] * 2u;
                    c |= 1ull << v;
                }
                E0[w] = (int)e;
#pragma unroll
                for (int k = 0; k < IB; k++) G[w][k] = (int)g[k];
#pragma unroll
                for (int r = 0; r < kKeep; r++) Fm[w][r] = (int)fm[r];
                cfg0[w] = c;
            }

        } else {
            // long tasks (>= 2^13 blocks each): each walk evaluates its start directly
#pragma unroll
            for (int w = 0; w < kWalks; w++) {
                unsigned long long task = base + (unsigned long long)(tid * kWalks + w);
                active[w] = task < ntasks;
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
            inner_walk<IB>(pk, std::make_integer_sequence<int, IS - 1>{});
            const bool flag_lo = (pk.M & 0xffffu) <= thr16;
            const bool flag_hi = (pk.M >> 16) <= thr16;
            if (__any_sync(0xffffffffu, flag_lo || flag_hi)) {
                // the warp rescans its flagged walks one at a time, all lanes on each
#pragma unroll
                for (int w = 0; w < kWalks; w++) {
                    unsigned todo = __ballot_sync(0xffffffffu, active[w] && ((w & 1) ? flag_hi : flag_lo));
                    while (todo) {
                        const int src = __ffs(todo) - 1;
                        todo &= todo - 1u;
                        if (lane == src) {
#pragma unroll
                            for (int k = 0; k < IB; k++) s_Gw[warp][k] = G[w][k];
                        }
                        __syncwarp();
                        const unsigned e0 = (unsigned)__shfl_sync(0xffffffffu, E0[w], src);
                        const unsigned long long cb = __shfl_sync(0xffffffffu, cfg0[w], src) | cmid;
                        warp_rescan<IB>(p, s, &s_buf_count, e0 - (unsigned)s.T[0], s_Gw[warp], cb, tau_scr, tie_E,
                                        tie_C, lane);
                        __syncwarp();
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
                } else if (active[0] && active[1] && active[2] && active[3]) {
                    // the four walks differ only in the task spins a = walk_shift (walks 1, 3 at
                    // +1) and a + 1 (walks 2, 3): one field by the definition, the others from it
                    const int f0 = field_at(s, n, j, cfg0[0] | cmid);
                    const int* Jj = s.Jq + j * n;
                    const unsigned da = (unsigned)Jj[walk_shift] << 1, db = (unsigned)Jj[walk_shift + 1] << 1;
                    F[0] = f0;
                    F[1] = (int)((unsigned)f0 + da);
                    F[2] = (int)((unsigned)f0 + db);
                    F[3] = (int)((unsigned)f0 + da + db);
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
    if (ensure_smem(reinterpret_cast<const void*>(gray_kernel<10>), (size_t)(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, gray_kernel<10>, kGrayThreads, smem) != cudaSuccess)
        return 0;
    return blocks;
}

template <int IB>
cudaError_t launch_gray_ib(const GrayParams& p, int grid, cudaStream_t s)
{
    size_t smem = gray_smem_bytes(p.n, p.list_cap);
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(gray_kernel<IB>), (size_t)(gray_smem_bytes(kMaxN, p.list_cap)));
    if (e != cudaSuccess) return e;
    gray_kernel<IB><<<grid, kGrayThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

namespace {

// The increment table is one per device.  Searches on different streams are ordered through
// it: a launch waits for the previous enumeration kernel on this device (an event recorded
// after it) before overwriting the table.  Inside a stream capture that event cannot be
// waited on, so a captured search relies on the order of the graph's launches instead.
constexpr int kMaxDevices = 64;
std::mutex g_table_mutex;
cudaEvent_t g_table_free[kMaxDevices];

}  // namespace

cudaError_t launch_gray(const GrayParams& p, int grid, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    const bool ordered = cs == cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_table_mutex);
    if (ordered) {
        if (!g_table_free[dev]) {
            e = cudaEventCreateWithFlags(&g_table_free[dev], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        e = cudaStreamWaitEvent(s, g_table_free[dev], 0);
        if (e != cudaSuccess) return e;
    }
    const void* table = reinterpret_cast<const char*>(p.prep) + offsetof(Prep, L) + offsetof(PrepLaunch, dT16);
    e = cudaMemcpyToSymbolAsync(c_dT16, table, sizeof(c_dT16), 0, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = p.inner_bits == 10 ? launch_gray_ib<10>(p, grid, s) : launch_gray_ib<9>(p, grid, s);
    if (e != cudaSuccess) return e;
    return ordered ? cudaEventRecord(g_table_free[dev], s) : cudaSuccess;
}

}  // namespace bf
