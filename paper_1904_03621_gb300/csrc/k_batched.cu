// Batched search (step A6): thousands of independent instances of uneven n
// in one persistent launch over an (instance, chunk) work queue.
//
// Every instance gets the single-instance treatment of k_prep.cu / k_gray.cu
// (exact fixed point, Gray walk with the two-lane 16-bit pre-filter, exact
// rescans), with these changes so that the whole sequence needs no host
// synchronisation and can be captured in a CUDA graph:
//   - the per-instance inner increments live in shared memory, loaded once per
//     work unit and read with 128-bit loads (LSU pipe) instead of kernel
//     parameters;
//   - a work unit is one block: 256 threads x 4 walks = 1024 tasks of
//     2^(9+m) configurations; blocks pop units from a queue of waves (unit w
//     of every instance, instances by decreasing n), and a barrier after every
//     unrolled block keeps the block's warps on the same stretch of code
//     (independent warps stalled on instruction fetch); warp 0 evaluates the
//     unit's common start once and every thread reaches its walks by a few
//     flips;
//   - each walk keeps one running 16-bit minimum per eighth of the block; hits
//     are collected warp-cooperatively: the flagged eighths of a walk are
//     rescanned by all 32 lanes (2 configurations each) into a bounded per-warp
//     buffer that is merged (warp bitonic sort, keep rule) before it can
//     overflow, so no spill area is needed;
//   - each unit appends its surviving records to the instance's pool and
//     lowers the instance threshold with atomicMin; a final kernel reselects
//     each instance's S lowest (float instances: re-evaluated as the quantised
//     energy plus the rounding residuals in 64-bit fixed point);
//   - zero-field instances (h = 0) walk the half space with the top spin at -1
//     (Z2 symmetry); the final kernel adds the mirrors.
#include <cfloat>
#include <climits>
#include <utility>

#include "bf_internal.cuh"
#include "bf_sort.cuh"
#include "bf_walk.cuh"

namespace bf {
namespace {

constexpr int kBWarps = 8;                    // warps per block of the walker
constexpr int kBThreads = kBWarps * 32;
constexpr int kBUnitWalkBits = 10;            // a work unit: 2^10 walks (256 threads x 4)
constexpr int kBBuf = 1024;                  // records per warp buffer (merged before a 32-record chunk could overflow it)
constexpr int kBKeepMax = kBBuf / 2;         // records a merged buffer may keep (S plus the float window)
constexpr int kBSeed = 1024;                  // sampled configurations per instance for its first threshold
constexpr int kBSampleMaxN = 10;              // largest n whose first threshold uses the sample
constexpr int kBPrepThreads = 256;
constexpr int kBDescents = 2;                 // local searches per warp of the preparation block
constexpr unsigned long long kBDescentSalt = 0x13198A2E03707344ull;
constexpr size_t kBWarpSmem = (size_t)kBBuf * 12;                 // record buffer bytes per warp
constexpr int kBSyncEvery = 1;                   // unrolled blocks between block barriers
// + the unit's tables: dT16, T (kBWalkSteps each), J_q (kBMaxN^2), h_q (kBMaxN), columns (kBMaxN x 16)
constexpr size_t kBSmem = kBWarpSmem * kBWarps + (size_t)kBWalkSteps * 8 + (size_t)kBMaxN * kBMaxN * 4 +
                          (size_t)kBMaxN * 4 + (size_t)kBMaxN * 16 * 4;

__device__ __forceinline__ double load_value(const void* p, int dtype, size_t idx)
{
    if (dtype == 0) return (double)static_cast<const int*>(p)[idx];
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

// sum over the block: warp shuffles, then one warp over the per-warp partial sums
__device__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// The k-th lowest (1 <= k <= kBMaxS) of the values the block's threads hold, kPer per thread
// (kEmptyE pads; kEmptyE when fewer than k are real).  Each warp extracts its k lowest by
// repeated warp minima, then warp 0 extracts the k-th lowest of the 8 sorted warp lists: two
// block barriers instead of a block-wide sort.
constexpr int kBPer = 4;                       // values per thread of kth_lowest
__device__ int kth_lowest(int (&v)[kBPer], int k, int* lists /* kBPrepThreads / 32 * kBMaxS */, int* out)
{
    // sort the thread's values ascending (insertion)
#pragma unroll
    for (int a = 1; a < kBPer; a++)
#pragma unroll
        for (int c = a; c > 0; c--)
            if (v[c] < v[c - 1]) { const int t = v[c]; v[c] = v[c - 1]; v[c - 1] = t; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int* L = lists + warp * kBMaxS;
    for (int r = 0; r < k; r++) {
        const int m = __reduce_min_sync(0xffffffffu, v[0]);
        const unsigned own = __ballot_sync(0xffffffffu, v[0] == m);
        if (lane == __ffs(own) - 1) {
#pragma unroll
            for (int a = 0; a + 1 < kBPer; a++) v[a] = v[a + 1];
            v[kBPer - 1] = kEmptyE;
        }
        if (lane == 0) L[r] = m;
    }
    __syncthreads();
    if (warp == 0) {
        constexpr int nw = kBPrepThreads / 32;
        int pos = 0, head = lane < nw ? lists[lane * kBMaxS] : kEmptyE, kth = kEmptyE;
        for (int r = 0; r < k; r++) {
            const int m = __reduce_min_sync(0xffffffffu, head);
            const unsigned own = __ballot_sync(0xffffffffu, head == m);
            if (lane == __ffs(own) - 1) {
                ++pos;
                head = pos < k ? lists[lane * kBMaxS + pos] : kEmptyE;
            }
            kth = m;
        }
        if (lane == 0) *out = kth;
    }
    __syncthreads();
    return *out;
}

// ---- per-instance preparation: one block per instance -----------------------

__global__ void __launch_bounds__(kBPrepThreads, 4) bprep_kernel(const BatchParams p)
{
    __shared__ double Jd[kBMaxN * kBMaxN];
    __shared__ double hd[kBMaxN];
    __shared__ double red[33];
    __shared__ int Jq[kBMaxN * kBMaxN];
    __shared__ int hq[kBMaxN];
    __shared__ int Tw[kBWalkSteps];                  // the walker's inner pair energies
    __shared__ int s_lists[kBPrepThreads / 32 * kBMaxS], s_kth;   // kth_lowest's warp lists
    __shared__ int s_z2;
    __shared__ int s_q, s_status, s_tau, s_dE[kBPrepThreads / 32], s_F[kBMaxN];
    __shared__ unsigned long long s_dC[kBPrepThreads / 32];
    __shared__ double s_emax;

    const int b = blockIdx.x, tid = threadIdx.x;
    BInst* I = p.inst + b;
    const int n = p.n[b];
    if (n < kBMinN || n > p.n_max || n > kBMaxN || (1ll << n) < p.S) {
        if (tid == 0) {
            I->n = n;
            I->n_full = n;
            I->z2 = 0;
            I->status = kErrArg;
            I->units = 0;
            atomicOr(&p.hdr->status, kErrArg);
            p.tau[b] = INT_MIN;
            p.pool_count[b] = 0u;
        }
        return;
    }
    const long long jo = p.J_off[b], ho = p.h_off[b];
    // one row of J per warp at a time, lane j = column j (n <= 32): the strict upper triangle
    const int lane = tid & 31, warp = tid >> 5;
    double part = 0.0;
    for (int i = warp; i < n; i += kBPrepThreads / 32) {
        const double x = (lane < n && i < lane) ? load_value(p.J, p.dtype, jo + (long long)i * n + lane) : 0.0;
        if (lane < n) Jd[i * n + lane] = x;
        part += fabs(x);
    }
    if (warp == 0 && lane < n) {
        hd[lane] = load_value(p.h, p.dtype, ho + lane);
        part += fabs(hd[lane]);
    }
    const double emax = block_sum(part, red);
    if (tid == 0) {
        int status = 0, q = 0;
        if (emax > 0.0) {
            int e;
            frexp(emax, &e);
            q = kEmqLog2 - e;
            if (p.dtype == 0) {
                if (q < 0) status |= kErrRange;
                q = q > 16 ? 16 : (q < 0 ? 0 : q);
            } else {
                q = q > 200 ? 200 : (q < -200 ? -200 : q);
            }
        }
        if (!(emax < 1e300)) status |= kErrRange;
        s_q = q;
        s_status = status;
        s_emax = emax;
    }
    __syncthreads();
    const int q = s_q;
    // J_q = rint(J 2^q), h_q = rint(h 2^q); 2^q is a power of two, so x 2^q is exact and so is
    // its distance to the rounded integer: the residual sum is accumulated in quantised units
    const double scale = ldexp(1.0, q);
    part = 0.0;
    for (int i = warp; i < n; i += kBPrepThreads / 32) {
        if (lane < n) {
            int v = 0;
            if (i < lane) {
                const double t = Jd[i * n + lane] * scale;
                const double r = rint(t);
                v = (int)r;
                part += fabs(t - r);
                // rho 2^(q+48) = (t - r) 2^48: t - r is exact (Sterbenz), the scaling too
                if (p.dtype != 0) I->R[i * n + lane] = __double2ll_rn(ldexp(t - r, kBResBits));
            }
            if (i <= lane) Jq[i * n + lane] = v;   // strict upper triangle and the diagonal (0)
            if (i < lane) Jq[lane * n + i] = v;    // mirrored into the lower triangle
        }
    }
    if (warp == 0 && lane < n) {
        const double t = hd[lane] * scale;
        const double r = rint(t);
        hq[lane] = (int)r;
        part += fabs(t - r);
        if (p.dtype != 0) I->Rh[lane] = __double2ll_rn(ldexp(t - r, kBResBits));
    }
    const double delta = ldexp(block_sum(part, red), -q);
    // zero fields: E(c) = E(~c), so the walker searches the half space with the top spin at -1
    // (an instance of n - 1 spins with fields h'_i = -J_{i,n-1}) and the final selection adds
    // each record's mirror.  The bound of the first threshold below stays valid: the distinct
    // configurations it ranks map to distinct configurations of the half space (c or ~c).
    if (warp == 0) {
        const bool hz = __all_sync(0xffffffffu, lane >= n || hd[lane] == 0.0);
        if (lane == 0) s_z2 = (hz && n - 1 >= kBMinN) ? 1 : 0;
    }
    static_assert(kBWalkBits <= kBMinN, "the walker's inner spins exist in every instance");
    // inner pair energies T[g] = sum_{i<k} J_ik s_i s_k over the walker's inner spins: the pairs
    // below the top inner spin by the definition, then T = t -+ f_top for the top spin at -1 / +1
    constexpr int kHalf = kBWalkSteps / 2, kTop = kBWalkBits - 1;
    for (int g = tid; g < kHalf; g += blockDim.x) {
        int t = 0, ft = 0;
        for (int i = 0; i < kTop; i++) {
            const int si = ((g >> i) & 1) ? 1 : -1;
            for (int k = i + 1; k < kTop; k++) t += Jq[i * n + k] * si * (((g >> k) & 1) ? 1 : -1);
            ft += Jq[i * n + kTop] * si;
        }
        Tw[g] = t - ft;
        Tw[g + kHalf] = t + ft;
    }
    __syncthreads();
    // first threshold.  n = 10: the S-th lowest of all 1024 exact energies.  Larger spaces take
    // the local search's bound below: a per-thread sampled walk (256 walks of 2^10
    // configurations) or an exact sample of 1024 configurations cost more preparation time
    // than their tighter start saved in the walker.
    const unsigned long long space = 1ull << n;
    const int filled = n > kBSampleMaxN ? 0 : (space < (unsigned long long)kBSeed ? (int)space : kBSeed);
    static_assert(kBSeed == kBPer * kBPrepThreads, "the sample is kBPer configurations per thread");
    {
        int ev[kBPer];
#pragma unroll
        for (int a = 0; a < kBPer; a++) {
            const int x = tid + a * kBPrepThreads;
            ev[a] = kEmptyE;
            if (x >= filled) continue;
            const unsigned long long c = (filled == (int)space) ? (unsigned long long)x
                                                                : (((unsigned long long)x * 0x9E3779B97F4A7C15ull) & (space - 1ull));
            int e = 0;
            for (int i = 0; i < n; i++) {
                int row = hq[i];
                for (int j = i + 1; j < n; j++) row += ((c >> j) & 1ull) ? Jq[i * n + j] : -Jq[i * n + j];
                e += ((c >> i) & 1ull) ? row : -row;
            }
            ev[a] = e;
        }
        // the S-th lowest sampled energy (of distinct configurations) bounds the S-th energy
        const int t = kth_lowest(ev, p.S, s_lists, &s_kth);
        if (tid == 0) s_tau = t;
    }

    // A second bound from a local search (n > 10; smaller spaces were enumerated above):
    // each warp runs steepest-descent searches from pseudo-random starts, lane l holding the
    // local field of spin l (flipping spin i changes Eq. (1) by -2 s_i f_i).  The S-th
    // lowest energy of the 1 + n + n(n-1)/2 distinct configurations within Hamming distance 2
    // of the best minimum bounds the S-th energy too; the lower of the two bounds is kept.
    const int ball = 1 + n + n * (n - 1) / 2;
    if (n > 10 && ball >= p.S) {
        int bE = kEmptyE;
        unsigned long long bC = kEmptyC;
        for (int r = 0; r < kBDescents; r++) {
            const unsigned long long id = ((unsigned long long)b * (kBPrepThreads / 32) + warp) * kBDescents + r;
            unsigned long long c = splitmix64(kBDescentSalt + id) & (space - 1ull);
            unsigned f = 0u;
            if (lane < n) {
                f = (unsigned)hq[lane];
                for (int j = 0; j < n; j++) {
                    const unsigned v = (unsigned)Jq[j * n + lane];
                    f += ((c >> j) & 1ull) ? v : 0u - v;
                }
            }
            unsigned t2 = 0u;
            if (lane < n) {
                const unsigned fh = f + (unsigned)hq[lane];
                t2 = ((c >> lane) & 1ull) ? fh : 0u - fh;
            }
            int E = (int)__reduce_add_sync(0xffffffffu, t2) >> 1;   // 2E = sum_i s_i (f_i + h_i)
            for (int it = 0; it < 4 * n; it++) {
                const int v = lane < n ? (((c >> lane) & 1ull) ? (int)f : -(int)f) : INT_MIN;
                const int best = __reduce_max_sync(0xffffffffu, v);
                if (best <= 0) break;
                const int k = __ffs(__ballot_sync(0xffffffffu, v == best)) - 1;
                c ^= 1ull << k;
                E -= 2 * best;
                if (lane < n) {
                    const unsigned d = (unsigned)Jq[k * n + lane] << 1;
                    f += ((c >> k) & 1ull) ? d : 0u - d;
                }
            }
            if (rec_less(E, c, bE, bC)) { bE = E; bC = c; }
        }
        if (lane == 0) { s_dE[warp] = bE; s_dC[warp] = bC; }
        __syncthreads();
        if (tid == 0) {
            for (int w2 = 1; w2 < kBPrepThreads / 32; w2++)
                if (rec_less(s_dE[w2], s_dC[w2], s_dE[0], s_dC[0])) { s_dE[0] = s_dE[w2]; s_dC[0] = s_dC[w2]; }
        }
        __syncthreads();
        const unsigned long long c0 = s_dC[0];
        const int E0 = s_dE[0];
        if (tid < n) {
            unsigned f = (unsigned)hq[tid];
            for (int j = 0; j < n; j++) {
                const unsigned v = (unsigned)Jq[j * n + tid];
                f += ((c0 >> j) & 1ull) ? v : 0u - v;
            }
            s_F[tid] = (int)f;
        }
        __syncthreads();
        // slots on a 32 x 32 grid, row i = warp + 8 a, column j = lane: (i, i) flips spin i,
        // (i, j) with i < j flips spins i and j, and (1, 0) is the minimum itself
        static_assert(kBPer * kBPrepThreads == kBMaxN * kBMaxN && kBPrepThreads == 8 * 32, "ball grid");
        int ev[kBPer];
#pragma unroll
        for (int a = 0; a < kBPer; a++) {
            const int i = warp + 8 * a, j = lane;
            ev[a] = kEmptyE;
            if (i == 1 && j == 0) {
                ev[a] = E0;
            } else if (i < n && j < n && i <= j) {
                const bool si = (c0 >> i) & 1ull;
                const unsigned fi = si ? (unsigned)s_F[i] : 0u - (unsigned)s_F[i];
                unsigned e = (unsigned)E0 - (fi << 1);
                if (i < j) {
                    const bool sj = (c0 >> j) & 1ull;
                    const unsigned fj = sj ? (unsigned)s_F[j] : 0u - (unsigned)s_F[j];
                    const unsigned jij = (unsigned)Jq[i * n + j] << 2;
                    e = e - (fj << 1) + (si == sj ? jij : 0u - jij);
                }
                ev[a] = (int)e;
            }
        }
        const int t = kth_lowest(ev, p.S, s_lists, &s_kth);
        if (tid == 0 && t < s_tau) s_tau = t;
    }
    __syncthreads();
    // outputs: the walked instance (n_w spins; the half space for zero fields)
    const int z2 = s_z2, nw = n - z2;
    for (int idx = tid; idx < nw * nw; idx += blockDim.x) I->Jq[idx] = Jq[(idx / nw) * n + idx % nw];
    for (int i = tid; i < kBMaxN; i += blockDim.x)
        I->hq[i] = i < nw ? (z2 ? -Jq[i * n + (n - 1)] : hq[i]) : 0;
    for (int g = tid; g < kBWalkSteps; g += blockDim.x) {
        I->T[g] = Tw[g];
        unsigned v = 0;
        if (g > 0) {
            int g1 = g ^ (g >> 1), g0 = (g - 1) ^ ((g - 1) >> 1);
            v = (unsigned)((Tw[g1] >> 16) - (Tw[g0] >> 16)) * 65537u;
        }
        I->dT16[g] = v;
    }
    for (int idx = tid; idx < kBMaxN * 16; idx += blockDim.x) {
        int j = idx / 16, k = idx % 16;
        int row = k < kBWalkBits + kKeep ? k : -1;
        I->col[j][k] = (j < nw && row >= 0 && row < nw) ? Jq[row * n + j] : 0;
    }
    if (tid == 0) {
        int status = s_status;
        int W = 0;
        if (p.dtype != 0 && delta > 0.0) {
            double eps = 8.0 * (double)n * (double)n * ldexp(1.0, -53) * s_emax;
            double w = ceil(ldexp(2.0 * delta + 2.0 * eps, q)) + 2.0;
            if (w > (double)(1 << 28)) { w = (double)(1 << 28); status |= kErrRange; }
            W = (int)w;
        }
        int m = nw - kBWalkBits - kBUnitWalkBits;   // 2^10 tasks per unit
        m = m < 0 ? 0 : (m > p.m_cap ? p.m_cap : m);
        const int nh = nw - kBWalkBits - m;
        I->n = nw;
        I->n_full = n;
        I->z2 = z2;
        I->q = q;
        I->W = W;
        I->m = m;
        I->nh = nh;
        I->status = status;
        I->units = nh > kBUnitWalkBits ? (1ull << (nh - kBUnitWalkBits)) : 1ull;
        I->delta = delta;
        I->emax = s_emax;
        p.tau[b] = s_tau;
        p.pool_count[b] = 0u;
        if (status) atomicOr(&p.hdr->status, (unsigned)status);
    }
}

// ---- work queue: instances ordered by decreasing n, unit prefix sums --------

constexpr int kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads) bplan_kernel(const BatchParams p)
{
    __shared__ unsigned cnt[kBMaxN + 1], start[kBMaxN + 1];
    const int tid = threadIdx.x;
    for (int i = tid; i <= kBMaxN; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    // counting sort by n, largest first; invalid instances (no units) go to bucket 0
    for (int b = tid; b < p.B; b += blockDim.x) {
        int n = p.inst[b].n;
        int key = (p.inst[b].status & kErrArg) ? 0 : n;
        atomicAdd(&cnt[key], 1u);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned s = 0;
        for (int n = kBMaxN; n >= 0; n--) { start[n] = s; s += cnt[n]; }
    }
    __syncthreads();
    for (int b = tid; b < p.B; b += blockDim.x) {
        int key = (p.inst[b].status & kErrArg) ? 0 : p.inst[b].n;
        unsigned pos = atomicAdd(&start[key], 1u);
        p.order[pos] = b;
    }
    __syncthreads();
    // waves: unit w of every instance that has more than w units, instances in queue order
    // (units are non-increasing along the order, so each wave is a prefix of it); a later
    // unit of an instance then starts from the threshold its earlier units produced
    __shared__ unsigned hist[64];
    for (int i = tid; i < 64; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (int k = tid; k < p.B; k += blockDim.x) {
        const unsigned long long un = p.inst[p.order[k]].units;
        if (un == 0) continue;
        atomicAdd(&hist[63 - __clzll(un)], 1u);          // units are powers of two
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long max_units = 0;
        for (int L = 0; L < 64; L++) if (hist[L]) max_units = 1ull << L;
        unsigned long long w_cap = (unsigned long long)p.max_waves;
        if (max_units > w_cap) { max_units = w_cap; atomicOr(&p.hdr->status, kErrArg); }
        unsigned long long run = 0, count = 0;
        for (int L = 0; L < 64; L++) count += hist[L];     // instances with >= 1 unit
        int L = 0;
        for (unsigned long long w = 0; w < max_units; w++) {
            while (L < 64 && (1ull << L) <= w) { count -= hist[L]; L++; }
            p.wave_off[w] = run;
            run += count;
        }
        p.wave_off[max_units] = run;
        p.hdr->task_next = 0ull;
        p.hdr->total_units = run;
        p.hdr->pad[0] = (unsigned)max_units;
    }
}

// ---- warp-level helpers ------------------------------------------------------

__device__ void warp_sort(int* E, unsigned long long* C, int len, int lane)
{
    for (int size = 2; size <= len; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncwarp();
            for (int i = lane; i < (len >> 1); i += 32) {
                int lo = ((i & -stride) << 1) + (i & (stride - 1));   // stride is a power of two
                cmp_swap(E, C, lo, lo + stride, (lo & size) == 0);
            }
        }
    }
    __syncwarp();
}

// Sort the buffer and keep the first S records (plus every record within W of the
// S-th for float instances).  Returns the new count; sets the S-th key when known.
__device__ int warp_merge(int* E, unsigned long long* C, int count, int S, int W, int& kE,
                          unsigned long long& kC, unsigned* status, int lane)
{
    int len = 64;
    while (len < count) len <<= 1;                   // count <= kBBuf
    for (int i = count + lane; i < len; i += 32) { E[i] = kEmptyE; C[i] = kEmptyC; }
    warp_sort(E, C, len, lane);
    if (count < S) return count;
    kE = E[S - 1];
    kC = C[S - 1];
    int keep = S;
    if (W > 0) {
        long long lim = (long long)kE + W;
        keep = upper_bound_key(E, len, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
        if (keep > count) keep = count;
        if (keep > kBKeepMax) {
            keep = kBKeepMax;
            if (lane == 0) atomicOr(status, kErrWindow);
        }
    }
    return keep;
}

// The running minimum is kept per eighth of the block (kBPart steps each): a flagged walk is
// rescanned only in the parts whose minimum reached the threshold.
constexpr int kBParts = 8;
constexpr int kBPart = kBWalkSteps / kBParts;
static_assert(kBPart % 32 == 0 && 2 * kBParts <= 32, "a part is whole Gray steps per lane; flags fit one word");

struct BPacked {
    unsigned Xa, Xb;
    unsigned M[kBParts];
    unsigned Ga[kBWalkBits], Gb[kBWalkBits];
};

template <int t>
__device__ __forceinline__ void bstep(BPacked& w, unsigned d)
{
    if constexpr (t > 0) {
        constexpr int k = cx_ctz(t);
        constexpr bool up = cx_up(t);
        constexpr int part = t / kBPart;
        w.Xa += (up ? w.Ga[k] : 0u - w.Ga[k]) + d;
        w.Xb += (up ? w.Gb[k] : 0u - w.Gb[k]) + d;
        if constexpr (t % kBPart == 0) w.M[part] = __vminu2(w.Xa, w.Xb);
        else w.M[part] = __vminu2(__vminu2(w.M[part], w.Xa), w.Xb);
    }
}

// four steps per 128-bit shared-memory load of the instance's increments
template <int g>
__device__ __forceinline__ void bwalk_group(BPacked& w, const uint4* tab4)
{
    const uint4 d = tab4[g];
    bstep<4 * g + 0>(w, d.x);
    bstep<4 * g + 1>(w, d.y);
    bstep<4 * g + 2>(w, d.z);
    bstep<4 * g + 3>(w, d.w);
}

template <int... Gs>
__device__ __forceinline__ void bwalk_block(BPacked& w, const uint4* tab4, std::integer_sequence<int, Gs...>)
{
    (bwalk_group<Gs>(w, tab4), ...);
}

}  // namespace

// ---- the persistent walker ------------------------------------------------------

__global__ void __launch_bounds__(kBThreads, 2) bwalk_kernel(const BatchParams p)
{
    // dynamic shared memory: per warp C[kBBuf], E[kBBuf]; then the unit's dT16[kBWalkSteps], T[kBWalkSteps]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long* Cw = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)wid * kBWarpSmem);
    int* Ew = reinterpret_cast<int*>(Cw + kBBuf);
    unsigned* dTw = reinterpret_cast<unsigned*>(smem_raw + kBWarpSmem * kBWarps);
    int* Tw = reinterpret_cast<int*>(dTw + kBWalkSteps);
    int* Jq = Tw + kBWalkSteps;                       // n x n (row stride n)
    int* hq = Jq + kBMaxN * kBMaxN;
    int (*colq)[16] = reinterpret_cast<int(*)[16]>(hq + kBMaxN);
    __shared__ unsigned long long s_unit;
    __shared__ int s_count[kBWarps];
    __shared__ int s_g[kBWarps][kBWalkBits];          // field row of the walk a warp is rescanning
    __shared__ int s_fc[kBMaxN], s_Gc[kBWalkBits], s_Ec;   // fields, inner fields, energy at the unit's cc
    const unsigned long long total = *(volatile unsigned long long*)&p.hdr->total_units;
    const int S = p.S;

    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(&p.hdr->task_next, 1ull);
        __syncthreads();
        const unsigned long long u = s_unit;
        if (u >= total) break;
        // wave w: wave_off[w] <= u < wave_off[w + 1]; the unit is unit w of the instance at
        // position u - wave_off[w] of the queue order
        int lo = 0, hi = (int)p.hdr->pad[0];
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (p.wave_off[mid] <= u) lo = mid; else hi = mid;
        }
        const int b = p.order[u - p.wave_off[lo]];
        const unsigned long long lu = (unsigned long long)lo;
        const BInst* I = p.inst + b;
        const int n = I->n, m = I->m, W = I->W;
        const unsigned long long ntasks = 1ull << I->nh;
        for (int i = threadIdx.x; i < kBWalkSteps; i += blockDim.x) {
            dTw[i] = I->dT16[i];
            Tw[i] = I->T[i];
        }
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) Jq[i] = I->Jq[i];
        for (int i = threadIdx.x; i < kBMaxN; i += blockDim.x) hq[i] = I->hq[i];
        for (int i = threadIdx.x; i < kBMaxN * 16; i += blockDim.x) colq[i / 16][i % 16] = I->col[i / 16][i % 16];
        __syncthreads();

        // The unit's common configuration cc has every task bit that differs between the block's
        // threads (bits 2..9 of the task index), both walk bits and all inner and middle spins at
        // -1.  Warp 0 evaluates its local fields and energy once; each thread reaches its first
        // walk from there by at most 8 flips, and the other three walks by one or two more.
        const int walk_shift = kBWalkBits + m;
        const unsigned long long cc = (lu << kBUnitWalkBits) << walk_shift;
        if (threadIdx.x < 32) {
            const int i = threadIdx.x;
            unsigned f = 0u, t2 = 0u;
            if (i < n) {
                f = (unsigned)hq[i];                          // f_i = h_i + sum_j J_ij s_j
                for (int j = 0; j < n; j++) {
                    const unsigned v = (unsigned)Jq[i * n + j];
                    f += ((cc >> j) & 1ull) ? v : 0u - v;
                }
                const unsigned fh = f + (unsigned)hq[i];
                t2 = ((cc >> i) & 1ull) ? fh : 0u - fh;      // 2E = sum_i s_i (f_i + h_i)
                s_fc[i] = (int)f;
                if (i < kBWalkBits) {
                    // G_i = 2 (h_i + sum_{j >= inner} J_ij s_j): f_i without the inner spins (all -1)
                    unsigned gi = f;
                    for (int j = 0; j < kBWalkBits; j++) gi += (unsigned)Jq[i * n + j];
                    s_Gc[i] = (int)(gi << 1);
                }
            }
            const unsigned e2 = __reduce_add_sync(0xffffffffu, t2);
            if (i == 0) s_Ec = (int)e2 >> 1;
        }
        __syncthreads();

        // walks of this thread: tasks lu * 2^10 + threadIdx.x * 4 + w
        int E0[kWalks], G[kWalks][kBWalkBits], Fm[kWalks][kKeep];
        unsigned long long cfg0[kWalks];
        unsigned active_mask = 0;
        const unsigned long long task0 = (lu << kBUnitWalkBits) + (unsigned long long)(threadIdx.x * kWalks);
#pragma unroll
        for (int w = 0; w < kWalks; w++)
            if (task0 + (unsigned long long)w < ntasks) active_mask |= 1u << w;
        // an inactive first walk (only in a unit of fewer than 2^10 tasks, where cc = 0) stays at cc
        const unsigned tb = (active_mask & 1u) ? (unsigned)threadIdx.x : 0u;
        cfg0[0] = cc | ((unsigned long long)tb << (walk_shift + 2));
        const int sa = walk_shift, sb = walk_shift + 1;        // the two walk bits
        {
            unsigned e = (unsigned)s_Ec;
            unsigned fa = sa < n ? (unsigned)s_fc[sa] : 0u, fb = sb < n ? (unsigned)s_fc[sb] : 0u;
            unsigned g0[kBWalkBits], fm0[kKeep];
#pragma unroll
            for (int k = 0; k < kBWalkBits; k++) g0[k] = (unsigned)s_Gc[k];
#pragma unroll
            for (int r = 0; r < kKeep; r++) fm0[r] = kBWalkBits + r < n ? (unsigned)s_fc[kBWalkBits + r] : 0u;
            // flip the thread's task spins from -1 to +1 in increasing order: E += 2 f_v, then every
            // field f_x += 2 J_xv (G_k by 4 J_kv)
            for (unsigned rest = tb; rest; rest &= rest - 1u) {
                const int v = walk_shift + 2 + (__ffs(rest) - 1);
                unsigned fv = (unsigned)s_fc[v];
                for (unsigned done = tb & ~rest; done; done &= done - 1u)
                    fv += (unsigned)Jq[(walk_shift + 2 + (__ffs(done) - 1)) * n + v] << 1;
                e += fv << 1;
#pragma unroll
                for (int k = 0; k < kBWalkBits; k++) g0[k] += (unsigned)Jq[k * n + v] << 2;
#pragma unroll
                for (int r = 0; r < kKeep; r++)
                    if (kBWalkBits + r < n) fm0[r] += (unsigned)Jq[(kBWalkBits + r) * n + v] << 1;
                if (sa < n) fa += (unsigned)Jq[sa * n + v] << 1;
                if (sb < n) fb += (unsigned)Jq[sb * n + v] << 1;
            }
            E0[0] = (int)e;
#pragma unroll
            for (int k = 0; k < kBWalkBits; k++) G[0][k] = (int)g0[k];
#pragma unroll
            for (int r = 0; r < kKeep; r++) Fm[0][r] = (int)fm0[r];
            // walk 1 = walk 0 with spin sa up; walk 2 = walk 0 with spin sb up; walk 3 = walk 1 with
            // spin sb up.  An inactive walk duplicates the walk it is copied from (an active walk's
            // spins sa / sb exist: its task index has that bit set)
#pragma unroll
            for (int w = 1; w < kWalks; w++) {
                const int from = (w == 3) ? 1 : 0;
                const int j = (w == 1) ? sa : sb;
                const bool act = (active_mask >> w) & 1u;
                cfg0[w] = act ? (cfg0[from] ^ (1ull << j)) : cfg0[from];
                unsigned fj = (w == 1) ? fa : fb;
                if (w == 3 && act) fj += (unsigned)Jq[sa * n + sb] << 1;   // field of sb once sa is up
                E0[w] = act ? (int)((unsigned)E0[from] + (fj << 1)) : E0[from];
#pragma unroll
                for (int k = 0; k < kBWalkBits; k++)
                    G[w][k] = act ? (int)((unsigned)G[from][k] + ((unsigned)Jq[k * n + j] << 2)) : G[from][k];
#pragma unroll
                for (int r = 0; r < kKeep; r++)
                    Fm[w][r] = (act && kBWalkBits + r < n)
                                   ? (int)((unsigned)Fm[from][r] + ((unsigned)Jq[(kBWalkBits + r) * n + j] << 1))
                                   : Fm[from][r];
            }
        }
        BPacked pk;
#pragma unroll
        for (int k = 0; k < kBWalkBits; k++) {
            pk.Ga[k] = pack_hi16(G[0][k], G[1][k]);
            pk.Gb[k] = pack_hi16(G[2][k], G[3][k]);
        }

        // per-warp record list (buffer) and threshold
        int count = 0, kE = kEmptyE;
        unsigned long long kC = kEmptyC;
        int tau_scr = 0;
        unsigned thr16 = 0;
        // tg: the instance threshold as read from global memory.  It only decreases, so every
        // value read is a valid bound and the lowest one read so far is the tightest.
        int tg_low = INT_MAX;
        auto refresh_with = [&](int tg) {
            tg_low = min(tg_low, tg);
            int t = min(tg_low, kE);
            long long ts = (long long)t + W;
            tau_scr = (int)(ts > (1ll << 30) ? (1ll << 30) : ts);
            thr16 = threshold16(tau_scr);
        };
        auto refresh = [&]() { refresh_with(*(volatile int*)&p.tau[b]); };
        refresh();
        unsigned long long cmid = 0ull;
        const unsigned nblocks = 1u << m;
        for (unsigned ub = 0; ub < nblocks; ++ub) {
            // every fourth block re-reads the instance threshold: the load is issued here and
            // consumed after the unrolled walk, so its latency is hidden
            const bool reread = (ub & 3u) == 3u;
            int tg_early = 0;
            if (reread) tg_early = *(volatile int*)&p.tau[b];
            pk.Xa = pack_energy(E0[0], E0[1]);
            pk.Xb = pack_energy(E0[2], E0[3]);
            pk.M[0] = __vminu2(pk.Xa, pk.Xb);
            bwalk_block(pk, reinterpret_cast<const uint4*>(dTw), std::make_integer_sequence<int, kBWalkSteps / 4>{});
            // one test of the minimum over the whole block first; the per-part flags (bit 2 part +
            // lane: the 16-bit lane whose minimum over that part reached the threshold; walks 0 and
            // 2 share lane 0, walks 1 and 3 lane 1) only when some lane of the warp is flagged
            unsigned mall = pk.M[0];
#pragma unroll
            for (int part = 1; part < kBParts; part++) mall = __vminu2(mall, pk.M[part]);
            const bool hit_any = (mall & 0xffffu) <= thr16 || (mall >> 16) <= thr16;
            const unsigned bal = __ballot_sync(0xffffffffu, hit_any);
            unsigned flags = 0u;
            if (bal) {
#pragma unroll
                for (int part = 0; part < kBParts; part++)
                    flags |= ((((pk.M[part] & 0xffffu) <= thr16) ? 1u : 0u) |
                              (((pk.M[part] >> 16) <= thr16) ? 2u : 0u))
                             << (2 * part);
            }
            if (bal) {
                // warp-cooperative exact rescan of every flagged walk
                for (unsigned rest = bal; rest; rest &= rest - 1u) {
                    const int L = __ffs(rest) - 1;
                    const unsigned fL = __shfl_sync(0xffffffffu, flags, L);
                    const unsigned aL = __shfl_sync(0xffffffffu, active_mask, L);
#pragma unroll
                    for (int w = 0; w < kWalks; w++) {
                        // this walk's lane in every part (bits 2 part)
                        const unsigned parts = (fL >> (w & 1)) & (0x55555555u >> (32 - 2 * kBParts));
                        if (!parts || !((aL >> w) & 1u)) continue;
                        const int e0 = __shfl_sync(0xffffffffu, E0[w], L);
                        if (lane == L) {
#pragma unroll
                            for (int k = 0; k < kBWalkBits; k++) s_g[wid][k] = G[w][k];
                        }
                        const unsigned long long cb = __shfl_sync(0xffffffffu, cfg0[w], L) | cmid;
                        __syncwarp();
                        // in each flagged part, lane l walks the Gray steps t = P + l R .. P + l R + R - 1:
                        // it sums the fields of its first configuration, then follows one flip per step
                        constexpr unsigned R = kBPart / 32;
                        const int* Gs = s_g[wid];
                        const unsigned base_e = (unsigned)e0 - (unsigned)Tw[0];
                        for (unsigned prest = parts; prest; prest &= prest - 1u) {
                        const unsigned part = (unsigned)(__ffs(prest) - 1) >> 1;
                        unsigned t = part * kBPart + (unsigned)lane * R;
                        unsigned g = t ^ (t >> 1);
                        unsigned sg = 0u;
#pragma unroll
                        for (int k = 0; k < kBWalkBits; k++) sg += ((g >> k) & 1u) ? (unsigned)Gs[k] : 0u;
#pragma unroll
                        for (unsigned i = 0; i < R; i++) {
                            if (count > kBBuf - 32) {
                                // room for the next 32 records: merge first (count is warp-uniform)
                                count = warp_merge(Ew, Cw, count, S, W, kE, kC, &p.hdr->status, lane);
                                if (count >= S && lane == 0) atomicMin(&p.tau[b], kE);
                                __syncwarp();
                                refresh();
                            }
                            if (i > 0) {
                                const int k = __ffs(++t) - 1;
                                g ^= 1u << k;
                                sg += ((g >> k) & 1u) ? (unsigned)Gs[k] : 0u - (unsigned)Gs[k];
                            }
                            const int e = (int)(base_e + (unsigned)Tw[g] + sg);
                            const unsigned long long c = cb | (unsigned long long)g;
                            const bool hit = e <= tau_scr && !(W == 0 && e == kE && c > kC);
                            const unsigned hb = __ballot_sync(0xffffffffu, hit);
                            if (hit) {
                                const int slot = count + __popc(hb & ((1u << lane) - 1u));
                                Ew[slot] = e;
                                Cw[slot] = c;
                            }
                            count += __popc(hb);
                        }
                        }
                        __syncwarp();
                    }
                }
                // tighten at once: the warp's S-th record bounds the instance's S-th energy
                if (count >= S) {
                    count = warp_merge(Ew, Cw, count, S, W, kE, kC, &p.hdr->status, lane);
                    if (lane == 0) atomicMin(&p.tau[b], kE);
                    __syncwarp();
                    refresh();
                }
            }
            if (reread) refresh_with(tg_early);
            if ((ub % kBSyncEvery) == kBSyncEvery - 1) __syncthreads();   // keep the warps on the same code
            // flip one middle spin
            if (ub + 1 < nblocks) {
                const unsigned u1 = ub + 1;
                const int jrel = __ffs(u1) - 1;
                const int j = kBWalkBits + jrel;
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
                } else if (active_mask == 0xfu) {
                    // the four walks differ only in the walk spins sa (walks 1, 3 at +1) and sb
                    // (walks 2, 3): one field by the definition, the others from it
                    const unsigned long long c = cfg0[0] | cmid;
                    int f = hq[j];
                    for (int i = 0; i < n; i++) f += ((c >> i) & 1ull) ? Jq[j * n + i] : -Jq[j * n + i];
                    const unsigned da = (unsigned)Jq[j * n + sa] << 1, db = (unsigned)Jq[j * n + sb] << 1;
                    F[0] = f;
                    F[1] = (int)((unsigned)f + da);
                    F[2] = (int)((unsigned)f + db);
                    F[3] = (int)((unsigned)f + da + db);
                } else {
#pragma unroll
                    for (int w = 0; w < kWalks; w++) {
                        const unsigned long long c = cfg0[w] | cmid;
                        int f = hq[j];
                        for (int i = 0; i < n; i++) f += ((c >> i) & 1ull) ? Jq[j * n + i] : -Jq[j * n + i];
                        F[w] = f;
                    }
                }
                int colv[kBWalkBits + kKeep];
#pragma unroll
                for (int k = 0; k < kBWalkBits + kKeep; k++) colv[k] = colq[j][k];
#pragma unroll
                for (int w = 0; w < kWalks; w++) {
                    const unsigned dE = (unsigned)F[w] << 1;
                    E0[w] = (int)((unsigned)E0[w] + (up ? dE : 0u - dE));
#pragma unroll
                    for (int k = 0; k < kBWalkBits; k++) {
                        const unsigned d = (unsigned)colv[k] << 2;
                        G[w][k] = (int)((unsigned)G[w][k] + (up ? d : 0u - d));
                    }
#pragma unroll
                    for (int r = 0; r < kKeep; r++) {
                        const unsigned d = (unsigned)colv[kBWalkBits + r] << 1;
                        Fm[w][r] = (int)((unsigned)Fm[w][r] + (up ? d : 0u - d));
                    }
                }
                cmid ^= 1ull << j;
#pragma unroll
                for (int k = 0; k < kBWalkBits; k++) {
                    pk.Ga[k] = pack_hi16(G[0][k], G[1][k]);
                    pk.Gb[k] = pack_hi16(G[2][k], G[3][k]);
                }
            }
        }
        // end of unit: every warp sorts its records, warp 0 merges the 8 lists and appends
        // the block's survivors to the instance pool (at most S plus the float window)
        if (count > 0) {
            count = warp_merge(Ew, Cw, count, S, W, kE, kC, &p.hdr->status, lane);
            if (count >= S && lane == 0) atomicMin(&p.tau[b], kE);
        }
        if (lane == 0) s_count[wid] = count;
        __syncthreads();
        if (wid == 0) {
            for (int w2 = 1; w2 < kBWarps; w2++) {
                const int cw = s_count[w2];
                if (cw == 0) continue;
                if (count + cw > kBBuf) {
                    count = warp_merge(Ew, Cw, count, S, W, kE, kC, &p.hdr->status, lane);
                    __syncwarp();
                }
                const unsigned long long* C2 =
                    reinterpret_cast<const unsigned long long*>(smem_raw + (size_t)w2 * kBWarpSmem);
                const int* E2 = reinterpret_cast<const int*>(C2 + kBBuf);
                for (int i = lane; i < cw; i += 32) {   // count, cw <= kBKeepMax after the merges: fits
                    Ew[count + i] = E2[i];
                    Cw[count + i] = C2[i];
                }
                count += cw;
                __syncwarp();
            }
            if (count > 0) {
                count = warp_merge(Ew, Cw, count, S, W, kE, kC, &p.hdr->status, lane);
                if (count >= S && lane == 0) atomicMin(&p.tau[b], kE);
                __syncwarp();
                const int tcur = min(*(volatile int*)&p.tau[b], kE);
                const long long lim = (long long)tcur + W;
                int keep = 0;   // the list is sorted: records up to the limit form a prefix
                for (int i = lane; i < count; i += 32) keep += ((long long)Ew[i] <= lim) ? 1 : 0;
                for (int o = 16; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
                unsigned base = 0;
                if (lane == 0 && keep > 0) base = atomicAdd(&p.pool_count[b], (unsigned)keep);
                base = __shfl_sync(0xffffffffu, base, 0);
                for (int i = lane; i < keep; i += 32) {
                    const unsigned slot = base + (unsigned)i;
                    if (slot < (unsigned)p.pool_cap) {
                        p.pool_E[(size_t)b * p.pool_cap + slot] = Ew[i];
                        p.pool_C[(size_t)b * p.pool_cap + slot] = Cw[i];
                    } else {
                        atomicOr(&p.hdr->status, kErrSpill);
                    }
                }
            }
        }
        __syncthreads();   // every warp is done with this unit's tables
    }
}

namespace {

// ---- per-instance final selection: one block per instance -----------------------

constexpr int kBFinalThreads = 128;

__global__ void __launch_bounds__(kBFinalThreads) bfinal_kernel(const BatchParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.x;
    const BInst* I = p.inst + b;
    const int len = p.final_len;                      // power of two >= pool_cap
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);
    int* E = reinterpret_cast<int*>(C + len);
    double* E64 = reinterpret_cast<double*>(E + len);  // aligned: len is a power of two >= 2
    __shared__ int s_keep;
    const int S = p.S;
    if (I->status & kErrArg) return;
    unsigned cnt = *(volatile unsigned*)&p.pool_count[b];
    if (cnt > (unsigned)p.pool_cap) cnt = p.pool_cap;
    // sort only the filled part of the pool (a power of two >= max(cnt, S))
    int lenb = 2;
    while (lenb < (int)cnt || lenb < S) lenb <<= 1;
    if (lenb > len) lenb = len;
    for (int i = threadIdx.x; i < lenb; i += blockDim.x) {
        bool ok = i < (int)cnt;
        E[i] = ok ? p.pool_E[(size_t)b * p.pool_cap + i] : kEmptyE;
        C[i] = ok ? p.pool_C[(size_t)b * p.pool_cap + i] : kEmptyC;
    }
    block_sort(E, C, lenb);
    if (threadIdx.x == 0) {
        int valid = upper_bound_key(E, lenb, INT_MAX - 1);
        int keep = valid < S ? valid : S;
        if (valid >= S && I->W > 0) {
            long long lim = (long long)E[S - 1] + I->W;
            keep = upper_bound_key(E, lenb, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
        }
        if (valid < S) atomicOr(&p.hdr->status, kErrSpill);   // cannot happen unless records were lost
        s_keep = keep;
    }
    __syncthreads();
    const int keep = s_keep;
    const int n = I->n_full;
    // Zero fields (I->z2): the records are the half space's lowest (top spin at -1).  With their
    // mirrors c ^ (2^n - 1), of the same energy, they contain the S lowest of the whole space: a
    // mirror's original precedes it in (E, c) order.  Within one energy level the half-space
    // records (c < 2^(n-1)) come first in increasing c, then the mirrors in the reverse order of
    // their originals.  One thread writes the S outputs from the sorted list (S <= 64).
    const unsigned long long mirror = (n >= 64 ? ~0ull : (1ull << n) - 1ull);
    auto emit_mirrored = [&](auto key_at, auto write) {
        int out = 0, i = 0;
        while (out < S && i < keep) {
            int j = i + 1;
            while (j < keep && key_at(j) == key_at(i)) j++;
            for (int t = i; t < j && out < S; t++) write(out++, t, 0ull);
            for (int t = j - 1; t >= i && out < S; t--) write(out++, t, mirror);
            i = j;
        }
        for (; out < S; out++) write(out, -1, 0ull);
    };
    if (p.dtype == 0) {
        if (I->z2) {
            if (threadIdx.x == 0)
                emit_mirrored([&](int t) { return E[t]; }, [&](int k, int t, unsigned long long x) {
                    static_cast<long long*>(p.energies)[(size_t)b * S + k] = t >= 0 ? (long long)(E[t] >> I->q) : LLONG_MAX;
                    p.states[(size_t)b * S + k] = t >= 0 ? C[t] ^ x : kEmptyC;
                });
            return;
        }
        for (int k = threadIdx.x; k < S; k += blockDim.x) {
            static_cast<long long*>(p.energies)[(size_t)b * S + k] = k < keep ? (long long)(E[k] >> I->q) : LLONG_MAX;
            p.states[(size_t)b * S + k] = C[k];
        }
        return;
    }
    // Re-evaluation of Eq. (1) for the kept records, then reselection by (E, c).  Eq. (1)
    // splits into the quantised energy and the rounding residuals, E(c) = 2^-q (E_q(c) + R(c)),
    // R(c) = sum_{i<j} rho_ij s_i s_j + sum_i rho_i s_i, summed exactly in 64-bit fixed point
    // (scale 2^(q+48), |rho'| <= 2^47 per term, at most 528 terms), then rounded once to FP64.
    // The residuals' truncation to that scale, at most 2^-(q+38) in all, lies far below the FP64
    // unit of E (emax 2^-29 ~ 2^-q).  Integer arithmetic instead of an FP64 sum per record: the
    // FP64 unit of this GPU issues 2 lanes per clock per SM.
    long long* Rs = reinterpret_cast<long long*>(E64 + len);   // n x n (row stride n), then h
    for (int x = threadIdx.x; x < n * n; x += blockDim.x) Rs[x] = (x % n > x / n) ? I->R[x] : 0ll;
    for (int x = threadIdx.x; x < n; x += blockDim.x) Rs[n * n + x] = I->Rh[x];
    int lenk = 2;                                      // a power of two >= max(keep, S), <= lenb
    while (lenk < keep || lenk < S) lenk <<= 1;
    if (lenk > lenb) lenk = lenb;
    __syncthreads();
    const double sq = ldexp(1.0, -I->q), sr = ldexp(1.0, -I->q - kBResBits);
    for (int r = threadIdx.x; r < lenk; r += blockDim.x) {
        if (r >= keep) {
            E64[r] = DBL_MAX;
            continue;
        }
        const unsigned long long c = C[r];
        long long R = 0;
        for (int i = 0; i < n; i++) {
            long long row = Rs[n * n + i];
            const long long* Ri = Rs + i * n;
            for (int j = i + 1; j < n; j++) row += ((c >> j) & 1ull) ? Ri[j] : -Ri[j];
            R += ((c >> i) & 1ull) ? row : -row;
        }
        E64[r] = (double)E[r] * sq + (double)R * sr;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < lenk; i += blockDim.x)
        if (i >= keep) C[i] = kEmptyC;
    block_sort(E64, C, lenk);
    if (I->z2) {
        if (threadIdx.x == 0)
            emit_mirrored([&](int t) { return E64[t]; }, [&](int k, int t, unsigned long long x) {
                static_cast<double*>(p.energies)[(size_t)b * S + k] = t >= 0 ? E64[t] : DBL_MAX;
                p.states[(size_t)b * S + k] = t >= 0 ? C[t] ^ x : kEmptyC;
            });
        return;
    }
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        static_cast<double*>(p.energies)[(size_t)b * S + k] = E64[k];
        p.states[(size_t)b * S + k] = C[k];
    }
}

}  // namespace

int batched_walker_blocks_per_sm()
{
    int blocks = 0;
    const size_t smem = kBSmem;
    if (ensure_smem(reinterpret_cast<const void*>(bwalk_kernel), (size_t)(smem)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, bwalk_kernel, kBThreads, smem) != cudaSuccess) return 0;
    return blocks;
}

cudaError_t launch_batched(const BatchParams& p, int walker_grid, cudaStream_t s)
{
    bprep_kernel<<<p.B, kBPrepThreads, 0, s>>>(p);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bplan_kernel<<<1, kPlanThreads, 0, s>>>(p);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = ensure_smem(reinterpret_cast<const void*>(bwalk_kernel), (size_t)(kBSmem));
    if (e != cudaSuccess) return e;
    bwalk_kernel<<<walker_grid, kBThreads, kBSmem, s>>>(p);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t smem = (size_t)p.final_len * 20 + (size_t)(kBMaxN * kBMaxN + kBMaxN) * 8;
    e = ensure_smem(reinterpret_cast<const void*>(bfinal_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    bfinal_kernel<<<p.B, kBFinalThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
