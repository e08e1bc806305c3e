// Tensor-core screening (step A2): energies of 128 x 256 configurations per
// tcgen05.mma, threshold test on the accumulator in TMEM.
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
// dR(r) + delta; delta bounds the split residuals (<= 2^-17 |x| each), the FP32
// accumulation and the conversions (values are below 2^31 in magnitude).  A
// flagged row is rescanned exactly in int32 and only exact hits are recorded.
// Per outer flip j: E_base += 2 s_j F_j, dR(r) += 4 s_j GR_j(r), dQ(c) += 4 s_j GC_j(c)
// with table lookups; the next tile's MMA is issued before the current tile's
// epilogue (two TMEM accumulators, two B buffers).
#include <climits>
#include <cuda_bf16.h>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kTcThreads = 512;                          // 16 warps: 4 per TMEM lane group
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
    const unsigned long long t0 = globaltimer();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(addr), "r"(parity));
        if (done) return true;
        if ((long long)(globaltimer() - t0) > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ float min3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// minimum of 64 consecutive accumulator columns of this thread's TMEM lane (one load, one wait)
__device__ __forceinline__ float tmem_min64(uint32_t taddr)
{
    uint32_t r[64];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
                 "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
                 "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
                   "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
                   "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
                   "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
                   "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // 3-input minimum tree over 64 values: 21 + 7 + 2 + 1 instructions (+1)
    float a[22];
#pragma unroll
    for (int i = 0; i < 21; i++)
        a[i] = min3(__uint_as_float(r[3 * i]), __uint_as_float(r[3 * i + 1]), __uint_as_float(r[3 * i + 2]));
    a[21] = __uint_as_float(r[63]);
    float b[8];
#pragma unroll
    for (int i = 0; i < 7; i++) b[i] = min3(a[3 * i], a[3 * i + 1], a[3 * i + 2]);
    b[7] = a[21];
    return min3(min3(b[0], b[1], b[2]), min3(b[3], b[4], b[5]), fminf(b[6], b[7]));
}

struct TcSm {
    uint16_t* A;            // 128 x 16 BF16 (K-major tile)
    uint16_t* B[2];         // 256 x 16 BF16 each
    int* Bint;              // [7][256] integer cross coefficients
    int* GR;                // [m][128]
    int* GC;                // [m][256]
    int* dQ;                // [3][256] column terms of the last three tiles
    int* Fo;                // [2][kTcMaxWalk] fields of the walked outer spins
    int* Jq;                // n x n
    int* hq;                // kMaxN
    int* E;                 // 2 * cap
    unsigned long long* C;  // 2 * cap
};

__device__ __forceinline__ void tc_record(const TcParams& p, const TcSm& s, unsigned* buf_count, int e,
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

__device__ __forceinline__ int field_of(const TcSm& s, int n, int j, unsigned long long cfg)
{
    int f = s.hq[j];
    for (int i = 0; i < n; i++) f += ((cfg >> i) & 1ull) ? s.Jq[j * n + i] : -s.Jq[j * n + i];
    return f;
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 1) tc_kernel(const __grid_constant__ TcParams p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int n = p.n, m = p.m, cap = p.list_cap;
    TcSm s;
    unsigned char* q = smem_raw;
    s.A = reinterpret_cast<uint16_t*>(q);            q += kTcRows * 16 * 2;
    s.B[0] = reinterpret_cast<uint16_t*>(q);         q += kTcCols * 16 * 2;
    s.B[1] = reinterpret_cast<uint16_t*>(q);         q += kTcCols * 16 * 2;
    s.C = reinterpret_cast<unsigned long long*>(q);  q += (size_t)2 * cap * 8;
    s.E = reinterpret_cast<int*>(q);                 q += (size_t)2 * cap * 4;
    s.Bint = reinterpret_cast<int*>(q);              q += kTcRowBits * kTcCols * 4;
    s.GR = reinterpret_cast<int*>(q);                q += kTcMaxWalk * kTcRows * 4;
    s.GC = reinterpret_cast<int*>(q);                q += kTcMaxWalk * kTcCols * 4;
    s.dQ = reinterpret_cast<int*>(q);                q += 3 * kTcCols * 4;
    s.Fo = reinterpret_cast<int*>(q);                q += 2 * kTcMaxWalk * 4;
    s.hq = reinterpret_cast<int*>(q);                q += kMaxN * 4;
    s.Jq = reinterpret_cast<int*>(q);

    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ unsigned s_buf_count;
    __shared__ int s_list_count, s_kE, s_abort;
    __shared__ unsigned long long s_kC, s_task;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane;        // TMEM lane of this thread
    const int quarter = warp >> 2;                 // accumulator columns [64 quarter, 64 quarter + 64)
    const bool owns_col = tid < kTcCols;           // threads 0..255 maintain one column term each
    const int col = tid & (kTcCols - 1);
    const Prep* prep = p.prep;

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
        for (int bb = 0; bb < 2; bb++) {
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
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(&s_tmem)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[1])));
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
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                           ((uint32_t)(kTcRows >> 4) << 24);
    const uint64_t adesc = make_desc(smem_u32(s.A));
    const uint64_t bdesc0 = make_desc(smem_u32(s.B[0])), bdesc1 = make_desc(smem_u32(s.B[1]));
    uint32_t phase0 = 0u, phase1 = 0u;
    unsigned char* const Bb0 = reinterpret_cast<unsigned char*>(s.B[0]);
    unsigned char* const Bb1 = reinterpret_cast<unsigned char*>(s.B[1]);
    bool aborted = false;

    const int S = p.S, W = p.W;
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
    refresh();
    auto issue = [&](int b) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(tmem + (uint32_t)(b * kTcCols)), "l"(adesc), "l"(b ? bdesc1 : bdesc0), "r"(idesc), "r"(0));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mbar[b])));
    };

    const int walk_shift = kTcSpins + m;
    const unsigned ntiles = 1u << m;
    const unsigned seg_mask = (1u << p.seg_log2) - 1u;
    const float delta = (float)p.delta;

    for (;;) {
        if (tid == 0) s_task = atomicAdd(&p.hdr->task_next, 1ull);
        __syncthreads();
        const unsigned long long task = s_task;
        if (task >= p.ntasks || s_abort) break;
        const unsigned long long c0 = p.hiconst | (task << walk_shift);
        // exact state of the task's first tile (walked spins, R and C all at -1)
        int Eb = 0;
        for (int i = 0; i < n; i++) {
            int rw = s.hq[i];
            for (int j = i + 1; j < n; j++) rw += ((c0 >> j) & 1ull) ? s.Jq[i * n + j] : -s.Jq[i * n + j];
            Eb += ((c0 >> i) & 1ull) ? rw : -rw;
        }
        int dR = 0;       // row term of this thread's row
        for (int i = 0; i < kTcRowBits; i++) {
            if (!((row >> i) & 1)) continue;
            dR += 2 * field_of(s, n, i, c0);
            for (int i2 = i + 1; i2 < kTcRowBits; i2++)
                if ((row >> i2) & 1) dR += 4 * s.Jq[i * n + i2];
        }
        int dQ = 0;       // column term of this thread's column
        for (int j = 0; j < kTcColBits; j++) {
            if (!((col >> j) & 1)) continue;
            dQ += 2 * field_of(s, n, kTcRowBits + j, c0);
            for (int j2 = j + 1; j2 < kTcColBits; j2++)
                if ((col >> j2) & 1) dQ += 4 * s.Jq[(kTcRowBits + j) * n + kTcRowBits + j2];
        }
        if (tid < m) s.Fo[tid] = field_of(s, n, kTcSpins + tid, c0);
        if (owns_col) {
            s.dQ[col] = dQ;
            *reinterpret_cast<uint32_t*>(Bb0 + tile_off(col, 14)) = split_bf16(dQ);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && !aborted) issue(0);

        unsigned long long cmid = 0ull;   // walked outer spins of the current tile: gray(u) << 15
        for (unsigned u = 0; u < ntiles; ++u) {
            const int b = u & 1;
            int Eb_n = Eb, dR_n = dR, dQ_n = dQ;
            // ---- prepare and issue tile u + 1
            if (u + 1 < ntiles) {
                const unsigned u1 = u + 1;
                const int j = __ffs(u1) - 1;
                const bool up = ((u1 ^ (u1 >> 1)) >> j) & 1u;
                const int Fj = s.Fo[b * kTcMaxWalk + j];
                Eb_n = (int)((unsigned)Eb + (up ? (unsigned)Fj << 1 : 0u - ((unsigned)Fj << 1)));
                const unsigned gr = (unsigned)s.GR[j * kTcRows + row] << 2;
                dR_n = (int)((unsigned)dR + (up ? gr : 0u - gr));
                const unsigned gc = (unsigned)s.GC[j * kTcCols + col] << 2;
                dQ_n = (int)((unsigned)dQ + (up ? gc : 0u - gc));
                if (tid < m) {
                    const unsigned d = (unsigned)s.Jq[(kTcSpins + tid) * n + kTcSpins + j] << 1;
                    s.Fo[(b ^ 1) * kTcMaxWalk + tid] = (int)((unsigned)s.Fo[b * kTcMaxWalk + tid] + (up ? d : 0u - d));
                }
                if (owns_col) {
                    s.dQ[((u + 1) % 3) * kTcCols + col] = dQ_n;
                    *reinterpret_cast<uint32_t*>((b ? Bb0 : Bb1) + tile_off(col, 14)) = split_bf16(dQ_n);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (tid == 0 && !aborted) issue(b ^ 1);
            }
            // ---- epilogue of tile u
            bool ok = !aborted && mbar_wait(smem_u32(&mbar[b]), b ? phase1 : phase0);
            if (b) phase1 ^= 1u; else phase0 ^= 1u;
            if (!ok && !aborted) {
                aborted = true;
                s_abort = 1;
                atomicOr(&p.hdr->status, kErrTimeout);
            }
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * kTcCols + 64 * quarter);
                const float mn = tmem_min64(ta);
                const float thr = (float)((long long)tau_scr - (long long)Eb - (long long)dR) + delta;
                if (mn <= thr) {
                    // exact rescan of this thread's row and 64 columns
                    const int* dQt = s.dQ + (u % 3) * kTcCols;
                    const unsigned long long cb = c0 | cmid | (unsigned long long)row;
                    const unsigned base = (unsigned)Eb + (unsigned)dR;
                    for (int cc = 0; cc < 64; cc++) {
                        const int c = 64 * quarter + cc;
                        unsigned acc = base + (unsigned)dQt[c];
#pragma unroll
                        for (int i = 0; i < kTcRowBits; i++)
                            acc += ((row >> i) & 1) ? (unsigned)s.Bint[i * kTcCols + c] : 0u;
                        const int e = (int)acc;
                        const unsigned long long cfg = cb | ((unsigned long long)c << kTcRowBits);
                        if (e <= tau_scr && !(e == tie_E && cfg > tie_C)) tc_record(p, s, &s_buf_count, e, cfg);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            Eb = Eb_n;
            dR = dR_n;
            dQ = dQ_n;
            // ---- segment boundary: merge the buffer into the block list (as in gray_kernel)
            if ((u & seg_mask) == seg_mask || u < 8u || u + 1 == ntiles) {
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
                        }
                        s_list_count = keep;
                        s_buf_count = 0u;
                    }
                    __syncthreads();
                }
                refresh();
                if (s_abort) aborted = true;
            }
            if (u + 1 < ntiles) {
                const unsigned u1 = u + 1;
                cmid ^= 1ull << (kTcSpins + __ffs(u1) - 1);
            }
        }
    }

    // ---- release TMEM (no MMA is in flight: every issued tile was waited for or timed out)
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
    return (size_t)kTcRows * 16 * 2 + (size_t)2 * kTcCols * 16 * 2 + (size_t)2 * list_cap * 12 +
           (size_t)kTcRowBits * kTcCols * 4 + (size_t)kTcMaxWalk * kTcRows * 4 + (size_t)kTcMaxWalk * kTcCols * 4 +
           (size_t)3 * kTcCols * 4 + (size_t)2 * kTcMaxWalk * 4 + (size_t)kMaxN * 4 + (size_t)n * n * 4;
}

cudaError_t launch_tc(const TcParams& p, int grid, cudaStream_t s)
{
    // at least 116 KB so that a second block cannot share the SM: each block holds all 512 TMEM columns
    size_t smem = tc_smem_bytes(p.n, p.list_cap);
    if (smem < (size_t)116 * 1024) smem = (size_t)116 * 1024;
    cudaError_t e = cudaFuncSetAttribute(tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_kernel<<<grid, kTcThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
