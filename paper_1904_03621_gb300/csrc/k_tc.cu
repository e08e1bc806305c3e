// Tensor-core screening (step A2): energies of 128 x 256 configurations per
// tcgen05.mma, reduced to one minimum per TMEM lane by the loading unit.
//
// Spin roles in a configuration c (bit i = spin i):
//   R = spins [0, 7)    rows of a tile (128 patterns, q_i = bit i of the row)
//   C = spins [7, 15)   columns of a tile (256 patterns)
//   O = spins [15, n)   one tile per outer configuration; [15, 15+m) are walked in
//                       reflected Gray order inside a task, the rest is the task
//                       index (and the fixed bits of subspace mode).
// With q in {0, 1} (q = 1 for s = +1) the energy of Eq. (1) splits exactly as
//   E(o, r, c) = E_base(o) + dR_o(r) + dQ_o(c) + X(r, c),
//   X(r, c) = 4 sum_{i in R, j in C} J_ij q_i(r) q_j(c),
// where E_base is the energy with all of R and C at -1, and dR / dQ the
// changes from setting the row / column spins alone (their local fields
// are taken with the other block at -1).  X does not depend on o: it is a
// 128 x 256 x 7 product of a 0/1 matrix (exact in BF16) with integer
// coefficients B_i(c) = 4 sum_j J_ij q_j(c).  The MMA computes
//   D[r, c] = sum_i q_i(r) (hi_i(c) + lo_i(c)) + (hi(dQ_o(c)) + lo(dQ_o(c)))
// with every integer split into two BF16 numbers (K = 7 x 2 + 2 = 16), FP32
// accumulation in TMEM.  A row is flagged when min_c D[r, c] <= tau - E_base -
// dR(r) + delta; delta bounds the split residuals (each <= 2^-16 |x|: two roundings to
// 8 significant bits; the split values of one product sum to less than 2^30 in magnitude,
// so less than 2^14 in all), the FP32 accumulation and the conversions (partial sums are
// below 2^31 in magnitude).  A
// flagged row is rescanned exactly in int32 and only exact hits are recorded.
// Per outer flip l: E_base += 2 s_l F_l, dR(r) += 4 s_l GR_l(r), dQ(c) += 4 s_l GC_l(c).
//
// Block = 8 epilogue warps + 2 MMA warps, no block-wide barrier inside a task:
//   * two TMEM accumulators (stages) of 256 columns, four B operands and four
//     row-base entries (tile t uses slot t mod 4);
//   * MMA warp s owns the tiles of stage s.  It follows the Gray walk of the
//     outer spins (E_base, the walked fields, 8 column terms and 4 row terms
//     per lane), waits `ready[s]`, issues the MMA, commits it to `full[s]` and
//     arrives on `full[s]` itself, then writes the dQ column of B and the row
//     bases E_base + dR(r) of its next tile (two ahead).  One committing
//     thread per stage: the commits of one thread complete in order, two
//     threads overlap;
//   * an epilogue warp waits `full[s]` (MMA done and its inputs published),
//     reads its row base, reads its 32 lanes x 128 columns with four
//     tcgen05.ld.red (minimum per lane) and arrives on `ready[s]`;
//   * candidate lists are merged every 2^seg tiles under a named barrier of
//     the epilogue warps only.
// Every wait is bounded; on a timeout the block stops issuing, flags
// kErrTimeout, waits for its last MMAs and frees its TMEM.
#include <climits>
#include <cuda_bf16.h>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kTcEpWarps = 8;                            // epilogue / operand warps
constexpr int kTcEpThreads = 32 * kTcEpWarps;            // 256
constexpr int kTcThreads = kTcEpThreads + 64;            // + one MMA warp per stage
constexpr int kTcBBufs = 4;                              // B operands in flight
constexpr int kTcRowBits = 7, kTcColBits = 8;
constexpr int kTcRows = 1 << kTcRowBits, kTcCols = 1 << kTcColBits;
constexpr int kTcSpins = kTcRowBits + kTcColBits;        // 15
constexpr int kTcMaxWalk = 16;                           // walked outer spins per task (max)
constexpr long long kTcWaitNs = 200000000ll;             // bounded waits: 0.2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; K-adjacent 8x16-byte core
// matrices 128 B apart (leading byte offset), 8-row groups 256 B apart (stride byte offset)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// byte offset of element (r, k) of a K-major 16-column BF16 tile in that layout
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// x ~ hi + lo in BF16 (round to nearest); returns hi in the low half (k even), lo in the high half
__device__ __forceinline__ uint32_t split_bf16(int x)
{
    const float xf = (float)x;
    const __nv_bfloat16 hi = __float2bfloat16_rn(xf);
    const __nv_bfloat16 lo = __float2bfloat16_rn(xf - __bfloat162float(hi));
    return (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for phase `parity` of an mbarrier; false after kTcWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(addr), "r"(parity) : "memory");
        if (done) return true;
        if ((long long)(globaltimer() - t0) > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(addr) : "memory");
}

// named barrier of the epilogue warps (the MMA warp does not take part)
__device__ __forceinline__ void ep_sync() { asm volatile("bar.sync 1, %0;" :: "n"(kTcEpThreads) : "memory"); }

// minimum over 128 consecutive accumulator columns of this thread's TMEM lane:
// four reducing loads of 32 columns and one wait, inside one asm block so that
// the loaded (unused) registers are private to it
__device__ __forceinline__ float tmem_min128(uint32_t taddr)
{
    float m0, m1, m2, m3;
    asm volatile("{\n\t.reg .b32 t<128>;\n\t"
                 "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 {t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15,t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31}, %0, [%4];\n\t"
                 "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 {t32,t33,t34,t35,t36,t37,t38,t39,t40,t41,t42,t43,t44,t45,t46,t47,t48,t49,t50,t51,t52,t53,t54,t55,t56,t57,t58,t59,t60,t61,t62,t63}, %1, [%5];\n\t"
                 "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 {t64,t65,t66,t67,t68,t69,t70,t71,t72,t73,t74,t75,t76,t77,t78,t79,t80,t81,t82,t83,t84,t85,t86,t87,t88,t89,t90,t91,t92,t93,t94,t95}, %2, [%6];\n\t"
                 "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 {t96,t97,t98,t99,t100,t101,t102,t103,t104,t105,t106,t107,t108,t109,t110,t111,t112,t113,t114,t115,t116,t117,t118,t119,t120,t121,t122,t123,t124,t125,t126,t127}, %3, [%7];\n\t"
                 "tcgen05.wait::ld.sync.aligned;\n\t}"
                 : "=f"(m0), "=f"(m1), "=f"(m2), "=f"(m3)
                 : "r"(taddr), "r"(taddr + 32u), "r"(taddr + 64u), "r"(taddr + 96u)
                 : "memory");
    return fminf(fminf(m0, m1), fminf(m2, m3));
}

struct TcSm {
    uint16_t* A;            // 128 x 16 BF16 (K-major tile)
    uint16_t* B[kTcBBufs];  // 256 x 16 BF16 each
    int* Bint;              // [7][256] integer cross coefficients
    int* GR;                // [m][128]
    int* GC;                // [m][256]
    int* dQ0;               // [2][256] column terms of the task's first tile (one copy per MMA warp)
    int* base;              // [4][128] E_base + dR(r) of the tiles in flight
    int* JW;                // [kTcMaxWalk][kTcMaxWalk] JW[l][l'] = J between walked spins l and l'
    int* Jq;                // n x n
    int* hq;                // kMaxN
    int* E;                 // 2 * cap
    unsigned long long* C;  // 2 * cap
};

__device__ __forceinline__ int field_of(const TcSm& s, int n, int j, unsigned long long cfg)
{
    int f = s.hq[j];
    for (int i = 0; i < n; i++) f += ((cfg >> i) & 1ull) ? s.Jq[j * n + i] : -s.Jq[j * n + i];
    return f;
}

// Exact rescan of one flagged row: the 128 columns [128 half, 128 half + 128)
// of the tile whose walked spins at +1 are the bits of g.  The column term of
// that tile is rebuilt from the task's first tile, dQ(c) = dQ0(c) + 4 sum_j
// q_j(c) sum_{l in g} J_{7+j,15+l}, so that only data written before the
// task's first barrier is read.
__device__ __noinline__ void tc_rescan(const TcParams& p, const int* Jq, const int* dQ0, const int* Bint, int* E,
                                       unsigned long long* C, unsigned* buf_count, int row, int half, unsigned base,
                                       unsigned g, unsigned long long c0, int tau_scr, int tie_E,
                                       unsigned long long tie_C)
{
    const int n = p.n, m = p.m;
    unsigned w4[kTcColBits];
#pragma unroll
    for (int j = 0; j < kTcColBits; j++) {
        unsigned a = 0u;
        for (int l = 0; l < m; l++)
            if ((g >> l) & 1u) a += (unsigned)Jq[(kTcRowBits + j) * n + kTcSpins + l];
        w4[j] = a << 2;
    }
    const unsigned long long cb = c0 | ((unsigned long long)g << kTcSpins) | (unsigned long long)row;
    for (int cc = 0; cc < 128; cc++) {
        const int c = 128 * half + cc;
        unsigned acc = base + (unsigned)dQ0[c];
#pragma unroll
        for (int j = 0; j < kTcColBits; j++) acc += ((c >> j) & 1) ? w4[j] : 0u;
#pragma unroll
        for (int i = 0; i < kTcRowBits; i++) acc += ((row >> i) & 1) ? (unsigned)Bint[i * kTcCols + c] : 0u;
        const int e = (int)acc;
        const unsigned long long cfg = cb | ((unsigned long long)c << kTcRowBits);
        if (e <= tau_scr && !(e == tie_E && cfg > tie_C)) {
            const unsigned slot = atomicAdd(buf_count, 1u);
            if (slot < (unsigned)p.list_cap) {
                E[p.list_cap + slot] = e;
                C[p.list_cap + slot] = cfg;
                continue;
            }
            const unsigned gs = atomicAdd(&p.hdr->spill_count, 1u);
            if (gs < p.spill_cap) {
                p.spill_E[gs] = e;
                p.spill_C[gs] = cfg;
            } else {
                atomicOr(&p.hdr->status, kErrSpill);
            }
        }
    }
}

// Gray step into tile v >= 1 of a task: walked spin l flips, up = it goes to +1
__device__ __forceinline__ void gray_step(unsigned v, int& l, bool& up)
{
    l = __ffs(v) - 1;
    up = (((v ^ (v >> 1)) >> l) & 1u) != 0u;
}

__device__ __forceinline__ unsigned addsub(unsigned x, unsigned d, bool up) { return up ? x + d : x - d; }

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 1) tc_kernel(const __grid_constant__ TcParams p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int n = p.n, m = p.m, cap = p.list_cap;
    TcSm s;
    unsigned char* q = smem_raw;
    s.A = reinterpret_cast<uint16_t*>(q);            q += kTcRows * 16 * 2;
    for (int b = 0; b < kTcBBufs; b++) {
        s.B[b] = reinterpret_cast<uint16_t*>(q);
        q += kTcCols * 16 * 2;
    }
    s.C = reinterpret_cast<unsigned long long*>(q);  q += (size_t)2 * cap * 8;
    s.E = reinterpret_cast<int*>(q);                 q += (size_t)2 * cap * 4;
    s.Bint = reinterpret_cast<int*>(q);              q += kTcRowBits * kTcCols * 4;
    s.GR = reinterpret_cast<int*>(q);                q += kTcMaxWalk * kTcRows * 4;
    s.GC = reinterpret_cast<int*>(q);                q += kTcMaxWalk * kTcCols * 4;
    s.dQ0 = reinterpret_cast<int*>(q);               q += 2 * kTcCols * 4;
    s.base = reinterpret_cast<int*>(q);              q += kTcBBufs * kTcRows * 4;
    s.JW = reinterpret_cast<int*>(q);                q += kTcMaxWalk * kTcMaxWalk * 4;
    s.hq = reinterpret_cast<int*>(q);                q += kMaxN * 4;
    s.Jq = reinterpret_cast<int*>(q);

    __shared__ __align__(8) unsigned long long full_bar[2], ready_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ unsigned s_buf_count;
    __shared__ int s_list_count, s_kE, s_abort;
    __shared__ unsigned long long s_kC, s_task;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
    __syncthreads();
    // constant operands: A (row patterns, ones) and the 14 cross columns of B (both buffers)
    for (int idx = tid; idx < kTcRows * 16; idx += blockDim.x) {
        const int r = idx >> 4, k = idx & 15;
        const float v = (k >= 2 * kTcRowBits) ? 1.0f : (float)((r >> (k >> 1)) & 1);
        s.A[tile_off(r, k) >> 1] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    for (int idx = tid; idx < kTcRowBits * kTcCols; idx += blockDim.x) {
        const int i = idx / kTcCols, c = idx % kTcCols;
        int b = 0;
        for (int j = 0; j < kTcColBits; j++)
            if ((c >> j) & 1) b += s.Jq[i * n + kTcRowBits + j];
        b *= 4;
        s.Bint[i * kTcCols + c] = b;
        const uint32_t pr = split_bf16(b);
        for (int bb = 0; bb < kTcBBufs; bb++) {
            s.B[bb][tile_off(c, 2 * i) >> 1] = (uint16_t)(pr & 0xffffu);
            s.B[bb][tile_off(c, 2 * i + 1) >> 1] = (uint16_t)(pr >> 16);
        }
    }
    // tables of the walked outer spins: GR_l(r) = sum_i J_{i,15+l} q_i(r), GC_l(c) = sum_j J_{7+j,15+l} q_j(c)
    for (int idx = tid; idx < m * kTcRows; idx += blockDim.x) {
        const int l = idx / kTcRows, r = idx % kTcRows;
        int g = 0;
        for (int i = 0; i < kTcRowBits; i++)
            if ((r >> i) & 1) g += s.Jq[i * n + kTcSpins + l];
        s.GR[l * kTcRows + r] = g;
    }
    for (int idx = tid; idx < m * kTcCols; idx += blockDim.x) {
        const int l = idx / kTcCols, c = idx % kTcCols;
        int g = 0;
        for (int j = 0; j < kTcColBits; j++)
            if ((c >> j) & 1) g += s.Jq[(kTcRowBits + j) * n + kTcSpins + l];
        s.GC[l * kTcCols + c] = g;
    }
    for (int idx = tid; idx < kTcMaxWalk * kTcMaxWalk; idx += blockDim.x) {
        const int l = idx / kTcMaxWalk, l2 = idx % kTcMaxWalk;
        s.JW[idx] = (l < m && l2 < m) ? s.Jq[(kTcSpins + l) * n + kTcSpins + l2] : 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(&s_tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" :: "r"(smem_u32(&full_bar[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&ready_bar[b])), "n"(kTcEpWarps));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_buf_count = 0u;
        s_list_count = 0;
        s_kE = kEmptyE;
        s_kC = kEmptyC;
        s_abort = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    const int S = p.S, W = prep->L.W;
    const int walk_shift = kTcSpins + m;
    const unsigned ntiles = 1u << m;
    const unsigned seg_mask = (1u << p.seg_log2) - 1u;
    const float delta = (float)p.delta;
    unsigned it0 = 0u;                 // global index of the task's first tile in this block
    bool aborted = false;

    // MMA warp state
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                           ((uint32_t)(kTcRows >> 4) << 24);
    long long last_issued = -1;        // last tile this MMA warp issued
    unsigned rph = 0u;                 // phases of ready[s] this MMA warp has waited for

    // epilogue warp state
    const int row = 32 * (warp & 3) + lane;        // TMEM lane of this thread
    const int half = (warp >> 2) & 1;              // accumulator columns [128 half, 128 half + 128)
    int tau_scr = 0, tie_E = kEmptyE;
    unsigned long long tie_C = kEmptyC;
    auto refresh = [&]() {
        const int tg = *(volatile int*)&p.hdr->tau;
        const int t = min(s_kE, tg);
        long long ts = (long long)t + W;
        tau_scr = (int)(ts > (1ll << 30) ? (1ll << 30) : ts);
        tie_E = (W == 0) ? s_kE : kEmptyE;
        tie_C = s_kC;
    };

    for (;;) {
        if (tid == 0) s_task = atomicAdd(&p.hdr->task_next, 1ull);
        __syncthreads();
        const unsigned long long task = s_task;
        const bool stop = task >= p.ntasks || s_abort;
        __syncthreads();
        if (stop) break;
        const unsigned long long c0 = p.hiconst | (task << walk_shift);

        if (warp >= kTcEpWarps) {
            // ---------------- MMA warp mst: Gray walk of the outer spins, operands and issue of stage mst
            const unsigned mst = (unsigned)(warp - kTcEpWarps);
            // exact energy of the task's first tile (R, C and walked spins at -1)
            int part = 0;
            for (int i = lane; i < n; i += 32) {
                int rw = s.hq[i];
                for (int j = i + 1; j < n; j++) rw += ((c0 >> j) & 1ull) ? s.Jq[i * n + j] : -s.Jq[i * n + j];
                part += ((c0 >> i) & 1ull) ? rw : -rw;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            int Eb = part;
            int Fo = lane < m ? field_of(s, n, kTcSpins + lane, c0) : 0;   // field of walked spin `lane`
            const int Fi = lane < kTcSpins ? field_of(s, n, lane, c0) : 0;  // field of tile spin `lane`
            int F[kTcSpins];
#pragma unroll
            for (int i = 0; i < kTcSpins; i++) F[i] = __shfl_sync(0xffffffffu, Fi, i);
            int dQ[kTcCols / 32], dR[kTcRows / 32];  // terms of columns / rows lane + 32 k
#pragma unroll
            for (int k = 0; k < kTcCols / 32; k++) {
                const int c = lane + 32 * k;
                int v = 0;
#pragma unroll
                for (int j = 0; j < kTcColBits; j++) {
                    if (!((c >> j) & 1)) continue;
                    v += 2 * F[kTcRowBits + j];
                    for (int j2 = j + 1; j2 < kTcColBits; j2++)
                        if ((c >> j2) & 1) v += 4 * s.Jq[(kTcRowBits + j) * n + kTcRowBits + j2];
                }
                dQ[k] = v;
                s.dQ0[mst * kTcCols + c] = v;
            }
#pragma unroll
            for (int k = 0; k < kTcRows / 32; k++) {
                const int r = lane + 32 * k;
                int v = 0;
#pragma unroll
                for (int i = 0; i < kTcRowBits; i++) {
                    if (!((r >> i) & 1)) continue;
                    v += 2 * F[i];
                    for (int i2 = i + 1; i2 < kTcRowBits; i2++)
                        if ((r >> i2) & 1) v += 4 * s.Jq[i * n + i2];
                }
                dR[k] = v;
            }
            // one step of the walk into tile v of the task
            auto step = [&](unsigned v) {
                int l; bool up;
                gray_step(v, l, up);
                const int Fl = __shfl_sync(0xffffffffu, Fo, l);
                Eb = (int)addsub((unsigned)Eb, (unsigned)Fl << 1, up);
                Fo = (int)addsub((unsigned)Fo, (unsigned)s.JW[l * kTcMaxWalk + (lane & (kTcMaxWalk - 1))] << 1, up);
#pragma unroll
                for (int k = 0; k < kTcCols / 32; k++)
                    dQ[k] = (int)addsub((unsigned)dQ[k], (unsigned)s.GC[l * kTcCols + lane + 32 * k] << 2, up);
#pragma unroll
                for (int k = 0; k < kTcRows / 32; k++)
                    dR[k] = (int)addsub((unsigned)dR[k], (unsigned)s.GR[l * kTcRows + lane + 32 * k] << 2, up);
            };
            // operand column and row bases of the tile in slot `slot`
            auto publish = [&](unsigned slot) {
                unsigned char* Bb = reinterpret_cast<unsigned char*>(s.B[slot]);
#pragma unroll
                for (int k = 0; k < kTcCols / 32; k++)
                    *reinterpret_cast<uint32_t*>(Bb + tile_off(lane + 32 * k, 14)) = split_bf16(dQ[k]);
#pragma unroll
                for (int k = 0; k < kTcRows / 32; k++)
                    s.base[slot * kTcRows + lane + 32 * k] = (int)((unsigned)Eb + (unsigned)dR[k]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            };
            unsigned u = (mst - it0) & 1u;             // first tile of this stage in the task
            if (p.stall_test) u = ntiles;              // testing only: issue nothing
            if (u < ntiles) {
                if (u == 1u) step(1u);
                publish((it0 + u) & (kTcBBufs - 1));
            }
            __syncwarp();
            bool first = true;
            const uint64_t adesc = make_desc(smem_u32(s.A));
            const uint32_t bsm0 = smem_u32(s.B[0]), bstride = smem_u32(s.B[1]) - bsm0;
            for (; u < ntiles; u += 2u) {
                const unsigned it = it0 + u;
                if (!aborted) aborted = __any_sync(0xffffffffu, *(volatile int*)&s_abort != 0);
                if (aborted) break;
                const bool more = u + 2u < ntiles;
                if (!first) {
                    // TMEM stage drained by the epilogue (tile u - 2)
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ready_bar[mst]), rph & 1u));
                    rph++;
                    if (!ok) {
                        aborted = true;
                        if (lane == 0) {
                            s_abort = 1;
                            atomicOr(&p.hdr->status, kErrTimeout);
                        }
                        break;
                    }
                }
                first = false;
                if (lane == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t bd = make_desc(bsm0 + (it & (kTcBBufs - 1)) * bstride);
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 :: "r"(tmem + mst * (uint32_t)kTcCols), "l"(adesc), "l"(bd), "r"(idesc), "r"(0));
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&full_bar[mst])) : "memory");
                    mbar_arrive(smem_u32(&full_bar[mst]));   // releases the row bases of tile u
                }
                last_issued = it;
                // the next tile of this stage: its B slot was last read by the MMA of tile u - 2,
                // complete since the epilogue drained that tile
                if (more) {
                    step(u + 1u);
                    step(u + 2u);
                    publish((it + 2u) & (kTcBBufs - 1));
                }
                __syncwarp();
            }
            it0 += ntiles;
            continue;
        }

        // ---------------- epilogue warps
        refresh();
        for (unsigned u = 0; u < ntiles; ++u) {
            const unsigned it = it0 + u, st = it & 1u;
            if (!aborted) aborted = __any_sync(0xffffffffu, *(volatile int*)&s_abort != 0);
            float mn = __int_as_float(0x7f800000);      // +inf
            int base = 0;
            if (!aborted) {
                const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&full_bar[st]), (it >> 1) & 1u));
                if (!ok) {
                    aborted = true;
                    if (lane == 0) {
                        s_abort = 1;
                        atomicOr(&p.hdr->status, kErrTimeout);
                    }
                } else {
                    base = s.base[(it & (kTcBBufs - 1)) * kTcRows + row];
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    mn = tmem_min128(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + st * (uint32_t)kTcCols +
                                     (uint32_t)(128 * half));
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                }
            }
            // stage st drained: the MMA of tile u + 2 may overwrite it
            __syncwarp();
            if (u + 2u < ntiles && lane == 0 && !aborted) mbar_arrive(smem_u32(&ready_bar[st]));
            // threshold test of this row; exact rescan of its 128 columns when flagged
            const float thr = (float)(int)((unsigned)tau_scr - (unsigned)base) + delta;
            if (mn <= thr)
                tc_rescan(p, s.Jq, s.dQ0 + st * kTcCols, s.Bint, s.E, s.C, &s_buf_count, row, half, (unsigned)base,
                          u ^ (u >> 1), c0, tau_scr, tie_E, tie_C);
            // segment boundary: merge the buffer into the block list
            if ((u & seg_mask) == seg_mask || u < 8u || u + 1u == ntiles) {
                ep_sync();
                const unsigned bc = s_buf_count;
                ep_sync();
                if (bc > 0u) {
                    const int lc = s_list_count;
                    const int nb = bc < (unsigned)cap ? (int)bc : cap;
                    for (int i = tid; i < 2 * cap; i += kTcEpThreads) {
                        if ((i >= lc && i < cap) || i >= cap + nb) {
                            s.E[i] = kEmptyE;
                            s.C[i] = kEmptyC;
                        }
                    }
                    group_sort(s.E, s.C, 2 * cap, tid, kTcEpThreads, [] { ep_sync(); });
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
                        }
                        s_list_count = keep;
                        s_buf_count = 0u;
                    }
                    ep_sync();
                }
                refresh();
            }
        }
        it0 += ntiles;
    }

    // ---- release TMEM once no MMA of this block is in flight
    if (warp >= kTcEpWarps && lane == 0 && last_issued >= 0 &&
        !mbar_wait(smem_u32(&full_bar[warp - kTcEpWarps]), ((unsigned)last_issued >> 1) & 1u))
        atomicOr(&p.hdr->status, kErrTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem));
    const int lc = s_list_count;
    for (int i = tid; i < cap; i += blockDim.x) {
        p.list_E[(size_t)blockIdx.x * cap + i] = i < lc ? s.E[i] : kEmptyE;
        p.list_C[(size_t)blockIdx.x * cap + i] = i < lc ? s.C[i] : kEmptyC;
    }
}

size_t tc_smem_bytes(int n, int list_cap)
{
    return (size_t)kTcRows * 16 * 2 + (size_t)kTcBBufs * kTcCols * 16 * 2 + (size_t)2 * list_cap * 12 +
           (size_t)kTcRowBits * kTcCols * 4 + (size_t)kTcMaxWalk * kTcRows * 4 + (size_t)kTcMaxWalk * kTcCols * 4 +
           (size_t)2 * kTcCols * 4 + (size_t)kTcBBufs * kTcRows * 4 + (size_t)kTcMaxWalk * kTcMaxWalk * 4 +
           (size_t)kMaxN * 4 + (size_t)n * n * 4;
}

cudaError_t launch_tc(const TcParams& p, int grid, cudaStream_t s)
{
    // at least 116 KB so that a second block cannot share the SM: each block holds all 512 TMEM columns
    size_t smem = tc_smem_bytes(p.n, p.list_cap);
    if (smem < (size_t)116 * 1024) smem = (size_t)116 * 1024;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(tc_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    tc_kernel<<<grid, kTcThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
