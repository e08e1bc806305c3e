// q-state Potts spin glass: the extension to other classical spin-glass
// models that Sec. 2 names (the Potts model of its Ref. Wu82).
//
// Model (sign as the library's Eq. (1)):
//     E(sigma) = sum_{i<j} J_ij [sigma_i == sigma_j] + sum_i h_i(sigma_i),
// sigma_i in {0, ..., q-1}, configuration integer c = sum_i sigma_i q^i (the
// base-q digits, generalising the binary coding of Sec. 3, Eq. (4)).  For
// q = 2, [s_i == s_j] = (1 + s_i s_j) / 2 and the model is an Ising instance.
//
// Digit layout of c:
//   [0, B)         inner digits: one fully unrolled block of q^B configurations
//                  in reflected q-ary Gray order (one digit changes by +-1 per step)
//   [B, B+m)       middle digits: walked in the same order, one change per block
//   [B+m, n)       task index (base q)
// Inside a block (outer digits o fixed):
//     E(x) = E_base(o) + sum_{k<B} (f_k(x_k) - f_k(0)) + T[x] - T[0],
//     f_k(v) = h_k(v) + sum_{l >= B} J_kl [v == sigma_l],
//     T[x] = sum_{k<k'<B} J_kk' [x_k == x_k'] ,
// so a step changing digit k from a to a +- 1 adds +-G_k(min(a, a')) + dT_t with
// G_k(v) = f_k(v+1) - f_k(v) and dT_t = T[x_t] - T[x_{t-1}].  The unrolled walk runs
// on 16-bit views of two walks packed in one register (see potts_walk_kernel): one
// IADD3 per step for both walks (kernel-parameter dT16 constants), one 3-input 16x2
// minimum per two steps.  A middle-digit change p: a -> a' shifts E_base by
// C_p(a') - C_p(a) + h_p(a') - h_p(a) (C_p(v) = sum_{l != p} J_pl [sigma_l == v], inner
// digits at 0) and updates four G entries per inner digit and two C entries per other
// middle digit (per-walk tables in shared memory).
//
// Arithmetic: exact int32 fixed point as for the Ising search (scale 2^qs,
// |E_q| <= 2^29, residual bound delta, window W, FP64 rescoring of float
// instances).  Selection, segments and the spill area follow gray_kernel.
#include <cfloat>
#include <climits>
#include <cstddef>
#include <mutex>
#include <type_traits>
#include <utility>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

// inner pair-table differences of the search being run (PottsPrep::dT, exact, and ::dT16, the
// 16-bit views in both lanes), copied in by launch_potts_walk; constant-bank operands of the walk
__constant__ int c_pdT[kPottsMaxSteps];
__constant__ unsigned c_pdT16[kPottsMaxSteps];

constexpr int kPottsThreads = 256;
constexpr int kPottsPrepThreads = 256;
constexpr int kPottsEmqLog2 = 29;

__device__ __forceinline__ double load_val(const void* p, int dtype, size_t idx)
{
    if (dtype == 0) return (double)static_cast<const int*>(p)[idx];
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

__device__ double block_sum_d(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// ---- prep: quantisation, residual bound, inner pair-table steps ----------------

__global__ void __launch_bounds__(kPottsPrepThreads) potts_prep_kernel(const void* J, const void* h, int n, int q,
                                                                       int dtype, PottsPrep* out, WsHeader* hdr)
{
    __shared__ double red[kPottsPrepThreads];
    __shared__ double s_Jd[kMaxN * kMaxN];
    __shared__ int s_q, s_status;
    __shared__ double s_emax;
    const int tid = threadIdx.x;
    const int B = potts_inner_digits(q);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        s_Jd[idx] = i < j ? load_val(J, dtype, idx) : 0.0;
    }
    __syncthreads();
    // emax = sum_{i<j} |J_ij| + sum_i max_v |h_i(v)| bounds |E| and every field difference / 2
    double part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) part += fabs(s_Jd[idx]);
    for (int i = tid; i < n; i += blockDim.x) {
        double mx = 0.0;
        for (int v = 0; v < q; v++) mx = fmax(mx, fabs(load_val(h, dtype, (size_t)i * q + v)));
        part += mx;
    }
    const double emax = block_sum_d(part, red);
    if (tid == 0) {
        int status = 0, qs = 0;
        if (emax > 0.0) {
            int e;
            frexp(emax, &e);                    // emax < 2^e
            qs = kPottsEmqLog2 - e;
            if (dtype == 0) {
                if (qs < 0) status |= kErrRange;
                if (qs > 16) qs = 16;
                if (qs < 0) qs = 0;
            } else {
                if (qs > 200) qs = 200;
                if (qs < -200) qs = -200;
            }
        }
        if (!(emax < 1e300)) status |= kErrRange;
        s_q = qs;
        s_status = status;
        s_emax = emax;
    }
    __syncthreads();
    const int qs = s_q;
    // quantise (symmetric, zero diagonal) and accumulate the residual bound
    part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        const int a = i < j ? i : j, b = i < j ? j : i;
        int v = 0;
        if (a != b) {
            const double x = s_Jd[a * n + b];
            const double r = rint(ldexp(x, qs));
            v = (int)r;
            if (i < j) part += fabs(x - ldexp(r, -qs));
        }
        out->Jq[idx] = v;
    }
    for (int i = tid; i < n; i += blockDim.x) {
        double mx = 0.0;
        for (int v = 0; v < q; v++) {
            const double x = load_val(h, dtype, (size_t)i * q + v);
            const double r = rint(ldexp(x, qs));
            out->hq[i * q + v] = (int)r;
            mx = fmax(mx, fabs(x - ldexp(r, -qs)));
        }
        part += mx;
    }
    const double delta = block_sum_d(part, red);
    __syncthreads();
    // dT_t = T[x_t] - T[x_{t-1}] over the inner Gray block (needs Jq: written above by this block)
    const int P = (int)potts_pow(q, B);
    for (int t = tid; t < kPottsMaxSteps; t += blockDim.x) {
        int d = 0, d16 = 0;
        if (t >= 1 && t < P && n >= B) {
            int T1 = 0, T0 = 0;
            for (int k = 0; k < B; k++)
                for (int k2 = k + 1; k2 < B; k2++) {
                    const int jv = out->Jq[k * n + k2];
                    if (potts_gray_digit(t, q, k) == potts_gray_digit(t, q, k2)) T1 += jv;
                    if (potts_gray_digit(t - 1, q, k) == potts_gray_digit(t - 1, q, k2)) T0 += jv;
                }
            d = T1 - T0;
            d16 = (T1 >> 16) - (T0 >> 16);           // floor(T / 2^16) differences telescope exactly
        }
        out->dT[t] = d;
        out->dT16[t] = (unsigned)d16 * 65537u;       // the same increment in both 16-bit lanes
    }
    if (tid == 0) {
        int status = s_status;
        int W = 0;
        if (dtype != 0 && delta > 0.0) {
            const double eps = 8.0 * (double)n * (double)n * ldexp(1.0, -53) * s_emax;
            double w = ceil(ldexp(2.0 * delta + 2.0 * eps, qs)) + 2.0;
            if (w > (double)(1 << 28)) { w = (double)(1 << 28); status |= kErrRange; }
            W = (int)w;
        }
        out->q = q;
        out->status = status;
        out->qs = qs;
        out->W = W;
        out->delta = delta;
        out->emax = s_emax;
        hdr->tau = INT_MAX;
        hdr->status = (unsigned)status;
        hdr->task_next = 0ull;
        hdr->spill_count = 0u;
    }
}

// exact quantised energy of configuration c (digits in base q)
__device__ int potts_energy_q(const int* Jq, const int* hq, int n, int q, unsigned long long c)
{
    unsigned char d[kMaxN];
    for (int i = 0; i < n; i++) {
        d[i] = (unsigned char)(c % (unsigned long long)q);
        c /= (unsigned long long)q;
    }
    unsigned e = 0u;
    for (int i = 0; i < n; i++) {
        e += (unsigned)hq[i * q + d[i]];
        const int* Ji = Jq + i * n;
        for (int j = i + 1; j < n; j++)
            if (d[i] == d[j]) e += (unsigned)Ji[j];
    }
    return (int)e;
}

// ---- seed: exact energies of a hashed sample -------------------------------------

constexpr int kPottsSeedThreads = 512;

__global__ void __launch_bounds__(kPottsSeedThreads) potts_seed_kernel(const PottsPrep* prep, int n, int q,
                                                                       unsigned long long space,
                                                                       unsigned long long sample, int per_block,
                                                                       int cap, int* outE, unsigned long long* outC)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);
    int* E = reinterpret_cast<int*>(C + per_block);
    int* Jq = E + per_block;
    int* hq = Jq + n * n;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Jq[i] = prep->Jq[i];
    for (int i = threadIdx.x; i < n * q; i += blockDim.x) hq[i] = prep->hq[i];
    __syncthreads();
    const bool full = sample >= space;        // whole space sampled: plain enumeration
    for (int k = threadIdx.x; k < per_block; k += blockDim.x) {
        const unsigned long long x = (unsigned long long)blockIdx.x * per_block + k;
        if (x >= sample || x >= space) { E[k] = kEmptyE; C[k] = kEmptyC; continue; }
        unsigned long long c = x;
        if (!full) {
            // splitmix64 of x, scaled onto [0, space)
            unsigned long long z = x + 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            c = __umul64hi(z, space);
        }
        E[k] = potts_energy_q(Jq, hq, n, q, c);
        C[k] = c;
    }
    block_sort(E, C, per_block);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        outE[(size_t)blockIdx.x * cap + i] = i < per_block ? E[i] : kEmptyE;
        outC[(size_t)blockIdx.x * cap + i] = i < per_block ? C[i] : kEmptyC;
    }
}

// ---- the walk ------------------------------------------------------------------

struct PottsSmem {
    int* Jq;                  // n*n
    int* hq;                  // n*q
    int* Gt;                  // [walk][B*Q][threads]: exact f_k(v) of each walk (fields of the inner digits)
    int* Ct;                  // [walk][m*Q][threads]: exact C_p(v) of each walk's middle digits
    int* E;                   // 2*cap
    unsigned long long* C;    // 2*cap
    int* step;                // q^B: Gray step t moves digit k from v to v+1 (or back): (k Q + v) << 1 | up
    int* xin;                 // q^B: inner configuration sum_k d_k q^k after step t
    int* mchg;                // q^m: the middle-digit change after block u: pm | a << 8 | a2 << 16
};

// integer packing hi * 2^16 + lo of two signed 16-bit increments
__device__ __forceinline__ unsigned pack2(int lo, int hi) { return ((unsigned)hi << 16) + (unsigned)lo; }

// 16-bit views floor((E + 2^31) / 2^16) of two energies in one register
__device__ __forceinline__ unsigned pack_e16(int lo, int hi)
{
    return (((unsigned)hi + 0x80000000u) & 0xffff0000u) | (((unsigned)lo + 0x80000000u) >> 16);
}

template <int Q, int B, int t>
__device__ __forceinline__ void potts_step(unsigned& X, unsigned& X1, unsigned& M, const unsigned (&G)[B][Q - 1],
                                           const PottsParams& p)
{
    constexpr int k = potts_qval(t, Q);
    constexpr int a0 = potts_gray_digit(t - 1, Q, k), a1 = potts_gray_digit(t, Q, k);
    constexpr bool up = a1 > a0;
    constexpr int v = up ? a0 : a1;
    X += (up ? G[k][v] : 0u - G[k][v]) + c_pdT16[t];
    if constexpr ((t & 1) != 0) {
        X1 = X;
    } else {
        M = __vminu2(__vminu2(M, X1), X);
    }
}

template <int Q, int B, int... Ts>
__device__ __forceinline__ void potts_block(unsigned& X, unsigned& X1, unsigned& M, const unsigned (&G)[B][Q - 1],
                                            const PottsParams& p, std::integer_sequence<int, Ts...>)
{
    (potts_step<Q, B, Ts + 1>(X, X1, M, G, p), ...);
}

__device__ __forceinline__ void potts_record(const PottsParams& p, const PottsSmem& s, unsigned* buf_count, int e,
                                             unsigned long long c)
{
    const unsigned slot = atomicAdd(buf_count, 1u);
    if (slot < (unsigned)p.list_cap) {
        s.E[p.list_cap + slot] = e;
        s.C[p.list_cap + slot] = c;
        return;
    }
    const unsigned g = atomicAdd(&p.hdr->spill_count, 1u);
    if (g < p.spill_cap) {
        p.spill_E[g] = e;
        p.spill_C[g] = c;
    } else {
        atomicOr(&p.hdr->status, kErrSpill);
    }
}

// 32-bit forms of the q-adic valuation and the reflected Gray digit for the block counter of
// the middle digits (q^m <= 256 blocks per task): division by the constant Q stays cheap.
template <int Q>
__device__ __forceinline__ int qval32(unsigned t)
{
    int k = 0;
    while (t % Q == 0u) { t /= Q; k++; }
    return k;
}

template <int Q>
__device__ __forceinline__ int gray_digit32(unsigned u, int pos)
{
    for (int i = 0; i < pos; i++) u /= Q;
    const int d = (int)(u % Q);
    return ((u / Q) & 1u) ? Q - 1 - d : d;
}

// Exact rescan of one walk's block by a whole warp.  Lane L takes the R = ceil(q^B / 32)
// Gray steps t = L*R .. L*R + R - 1.  It evaluates its first configuration directly:
//   E = Ebase + sum_k (f_k(d_k) - f_k(0)) - sum_{k<l<B} J_kl [d_k != d_l]
// (Ebase has all inner digits 0, so every inner pair is equal there), then follows the
// steps as the walk does: +-(f_k(v+1) - f_k(v)) for the changed digit plus the pair-table
// difference.  F points at the walk's field table f_k(v), entry k Q + v at F[(k Q + v) * threads].
template <int Q, int B>
__device__ __forceinline__ void potts_warp_rescan(const PottsParams& p, const PottsSmem& s, unsigned* buf_count,
                                                  unsigned ebase, const int* F, unsigned long long cb, int tau,
                                                  int tie_E, unsigned long long tie_C, int n, int lane)
{
    constexpr int P = (int)potts_pow(Q, B);
    constexpr int R = (P + 31) / 32;
    const int t0 = lane * R;
    if (t0 >= P) return;
    const int t1 = t0 + R < P ? t0 + R : P;
    int d[B];
    int x = s.xin[t0];
#pragma unroll
    for (int k = 0; k < B; k++) {
        d[k] = x % Q;
        x /= Q;
    }
    unsigned e = ebase;
#pragma unroll
    for (int k = 0; k < B; k++) {
        e += (unsigned)(F[(k * Q + d[k]) * kPottsThreads] - F[(k * Q) * kPottsThreads]);
#pragma unroll
        for (int l = k + 1; l < B; l++)
            if (d[k] != d[l]) e -= (unsigned)s.Jq[k * n + l];
    }
    for (int t = t0; t < t1; t++) {
        if (t > t0) {
            const int st = s.step[t], kv = st >> 1;
            const unsigned g = (unsigned)(F[(kv + 1) * kPottsThreads] - F[kv * kPottsThreads]);
            e += ((st & 1) ? g : 0u - g) + (unsigned)c_pdT[t];
        }
        const int ei = (int)e;
        const unsigned long long c = cb + (unsigned long long)s.xin[t];
        if (ei <= tau && !(ei == tie_E && c > tie_C)) potts_record(p, s, buf_count, ei, c);
    }
}

// Each thread walks two tasks at once: their 16-bit energy views share one register, so one
// IADD3 advances both and one 3-input 16x2 minimum folds two steps.  A digit's increment is
// the difference of the floors of its cumulative field offset F_k(v) = f_k(v) - f_k(0), so the
// views telescope exactly and, as for the Ising walk,
//     E/2^16 - (B + 2) < x - 2^15 <= E/2^16 + 1 ,
// and x <= floor((tau + 2^31) / 2^16) + 1 catches every E <= tau.  Flagged walks are
// rescanned exactly from their int32 tables, by the whole warp.
template <int Q>
__global__ void __launch_bounds__(kPottsThreads, 2) potts_walk_kernel(const __grid_constant__ PottsParams p)
{
    constexpr int B = potts_inner_digits(Q);
    constexpr int P = (int)potts_pow(Q, B);
    constexpr int NF = B * Q;                 // per-walk field table entries f_k(v)
    constexpr int NW = kPottsWalks;
    static_assert(NW == 2, "two walks: the two 16-bit lanes of one register");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = p.n, m = p.m, cap = p.list_cap;
    PottsSmem s;
    s.C = reinterpret_cast<unsigned long long*>(smem_raw);
    s.E = reinterpret_cast<int*>(s.C + 2 * cap);
    s.Gt = s.E + 2 * cap;
    s.Ct = s.Gt + NW * NF * kPottsThreads;
    s.Jq = s.Ct + NW * kPottsMidTable * kPottsThreads;
    s.hq = s.Jq + n * n;
    s.step = s.hq + n * Q;
    s.xin = s.step + P;
    s.mchg = s.xin + P;

    __shared__ unsigned s_buf_count;
    __shared__ int s_list_count, s_kE;
    __shared__ unsigned long long s_batch, s_kC;

    const int tid = threadIdx.x;
    const PottsPrep* prep = p.prep;
    if (*(volatile unsigned*)&p.hdr->status & kErrRange) {
        // the instance is outside the fixed-point range (reported by the workspace status): no walk
        for (int i = tid; i < cap; i += blockDim.x) {
            p.list_E[(size_t)blockIdx.x * cap + i] = kEmptyE;
            p.list_C[(size_t)blockIdx.x * cap + i] = kEmptyC;
        }
        return;
    }
    for (int i = tid; i < n * n; i += blockDim.x) s.Jq[i] = prep->Jq[i];
    for (int i = tid; i < n * Q; i += blockDim.x) s.hq[i] = prep->hq[i];
    for (int t = tid; t < P; t += blockDim.x) {
        int x = 0, qk = 1;
        for (int k = 0; k < B; k++, qk *= Q) x += potts_gray_digit((unsigned long long)t, Q, k) * qk;
        s.xin[t] = x;
        int st = 0;
        if (t > 0) {
            const int k = potts_qval((unsigned long long)t, Q);
            const int a0 = potts_gray_digit((unsigned long long)(t - 1), Q, k);
            const int a1 = potts_gray_digit((unsigned long long)t, Q, k);
            st = ((k * Q + (a1 > a0 ? a0 : a1)) << 1) | (a1 > a0 ? 1 : 0);
        }
        s.step[t] = st;
    }
    // the middle-digit change after block u (u + 1 < q^m <= kPottsMaxBlocks): the digit pm = the
    // q-adic valuation of u + 1 moves from a to a2, the same for every walk of the launch
    for (int u = tid; u + 1 < (int)p.qpow[p.m] && u < kPottsMaxBlocks; u += blockDim.x) {
        const int pm = qval32<Q>((unsigned)u + 1u);
        const int a = gray_digit32<Q>((unsigned)u, pm), a2 = gray_digit32<Q>((unsigned)u + 1u, pm);
        s.mchg[u] = pm | (a << 8) | (a2 << 16);
    }
    if (tid == 0) {
        s_buf_count = 0u;
        s_list_count = 0;
        s_kE = kEmptyE;
        s_kC = kEmptyC;
    }
    __syncthreads();

    const int S = p.S, W = prep->W;
    const unsigned long long nblocks = p.qpow[m];
    const unsigned long long seg_mask = (1ull << p.seg_log2) - 1ull;
    const unsigned long long task_mul = p.qpow[B + m];
    // entry e of walk w at table[(w * entries + e) * kPottsThreads]
    int* Gt = s.Gt + tid;
    int* Ct = s.Ct + tid;

    int tau_scr = 0, tie_E = kEmptyE;
    unsigned long long tie_C = kEmptyC;
    unsigned thr16 = 0u;
    auto refresh = [&]() {
        const int tg = *(volatile int*)&p.hdr->tau;
        const int t = min(s_kE, tg);
        tie_E = (W == 0) ? s_kE : kEmptyE;
        tie_C = s_kC;
        long long ts = (long long)t + W;
        if (ts > (1ll << 30)) ts = 1ll << 30;
        tau_scr = (int)ts;
        const unsigned th = (((unsigned)tau_scr + 0x80000000u) >> 16) + 1u;
        thr16 = th > 0xffffu ? 0xffffu : th;
    };
    refresh();

    for (;;) {
        if (tid == 0) s_batch = atomicAdd(&p.hdr->task_next, (unsigned long long)(NW * kPottsThreads));
        __syncthreads();
        const unsigned long long base = s_batch;
        __syncthreads();
        if (base >= p.ntasks) break;
        bool active[NW];
        unsigned long long c0[NW];
        unsigned Ebase[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) {
            unsigned long long task = base + (unsigned long long)(NW * tid + w);
            active[w] = task < p.ntasks;
            if (!active[w]) task = 0;               // a valid walk whose hits are ignored
            c0[w] = task * task_mul;
        }

        // ---- state at the start of the task (inner and middle digits 0), per walk
#pragma unroll 1
        for (int w = 0; w < NW; w++) {
            unsigned char d[kMaxN];
            unsigned long long x = c0[w];
            for (int i = 0; i < n; i++) {
                d[i] = (unsigned char)(x % (unsigned long long)Q);
                x /= (unsigned long long)Q;
            }
            unsigned e = 0u;
            for (int i = 0; i < n; i++) {
                e += (unsigned)s.hq[i * Q + d[i]];
                for (int j = i + 1; j < n; j++)
                    if (d[i] == d[j]) e += (unsigned)s.Jq[i * n + j];
            }
            Ebase[w] = e;
            // f_k(v) = h_k(v) + sum_{l >= B} J_kl [v == d_l] (fields of the inner digits from the rest)
            for (int k = 0; k < B; k++) {
                int f[Q];
#pragma unroll
                for (int v = 0; v < Q; v++) f[v] = s.hq[k * Q + v];
                for (int l = B; l < n; l++) {
                    const int jv = s.Jq[k * n + l];
#pragma unroll
                    for (int v = 0; v < Q; v++) f[v] += (d[l] == v) ? jv : 0;
                }
#pragma unroll
                for (int v = 0; v < Q; v++) Gt[(w * NF + k * Q + v) * kPottsThreads] = f[v];
            }
            // C_p(v) = sum_{l != B+p} J_{B+p, l} [d_l == v] for the middle digits
            for (int pm = 0; pm < m; pm++) {
                const int sp = B + pm;
                int cv[Q];
#pragma unroll
                for (int v = 0; v < Q; v++) cv[v] = 0;
                for (int l = 0; l < n; l++) {
                    if (l == sp) continue;
                    const int jv = s.Jq[sp * n + l];
#pragma unroll
                    for (int v = 0; v < Q; v++) cv[v] += (d[l] == v) ? jv : 0;
                }
#pragma unroll
                for (int v = 0; v < Q; v++) Ct[(w * kPottsMidTable + pm * Q + v) * kPottsThreads] = cv[v];
            }
        }

        for (unsigned long long u = 0; u < nblocks; ++u) {
            // ---- one block of q^B configurations for both walks
            unsigned G[B][Q - 1];
#pragma unroll
            for (int k = 0; k < B; k++) {
                // cumulative offsets F_k(v) = f_k(v) - f_k(0) of the two walks and their floors
                const int b0 = Gt[(0 * NF + k * Q) * kPottsThreads], b1 = Gt[(1 * NF + k * Q) * kPottsThreads];
                int h0 = 0, h1 = 0;                     // floor(F_k(v) / 2^16), F_k(0) = 0
#pragma unroll
                for (int v = 0; v < Q - 1; v++) {
                    const int n0 = (int)((unsigned)Gt[(0 * NF + k * Q + v + 1) * kPottsThreads] - (unsigned)b0) >> 16;
                    const int n1 = (int)((unsigned)Gt[(1 * NF + k * Q + v + 1) * kPottsThreads] - (unsigned)b1) >> 16;
                    G[k][v] = pack2(n0 - h0, n1 - h1);
                    h0 = n0;
                    h1 = n1;
                }
            }
            unsigned X = pack_e16((int)Ebase[0], (int)Ebase[1]);
            unsigned X1 = X, M = X;
            potts_block<Q, B>(X, X1, M, G, p, std::make_integer_sequence<int, P - 1>{});
            M = __vminu2(M, X1);
            const bool flag[NW] = {active[0] && (M & 0xffffu) <= thr16, active[1] && (M >> 16) <= thr16};
            if (__any_sync(0xffffffffu, flag[0] || flag[1])) {
                unsigned long long mid = 0ull;
                for (int pm = 0; pm < m; pm++) mid += (unsigned long long)gray_digit32<Q>((unsigned)u, pm) * p.qpow[pm];
                const unsigned long long midc = mid * p.qpow[B];
                const int lane = tid & 31;
#pragma unroll
                for (int w = 0; w < NW; w++) {
                    unsigned todo = __ballot_sync(0xffffffffu, flag[w]);
                    while (todo) {
                        const int src = __ffs(todo) - 1;
                        todo &= todo - 1u;
                        const unsigned eb = __shfl_sync(0xffffffffu, Ebase[w], src);
                        const unsigned long long cw = __shfl_sync(0xffffffffu, c0[w], src);
                        const int* Gs = s.Gt + (tid - lane + src) + w * NF * kPottsThreads;
                        potts_warp_rescan<Q, B>(p, s, &s_buf_count, eb, Gs, cw + midc, tau_scr, tie_E, tie_C, n,
                                                lane);
                    }
                }
                __syncwarp();   // the tables of other lanes were read: they change below
            }

            // ---- segment boundary: merge the buffer into the block list
            if ((u & seg_mask) == seg_mask || u < 16ull || u + 1 == nblocks) {
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
                                const long long lim = (long long)K + W;
                                keep = upper_bound_key(s.E, 2 * cap, lim > INT_MAX - 1 ? INT_MAX - 1 : (int)lim);
                                if (keep > total) keep = total;
                                if (keep > cap) { keep = cap; atomicOr(&p.hdr->status, kErrWindow); }
                            }
                            s_kE = K;
                            s_kC = s.C[S - 1];
                            atomicMin(&p.hdr->tau, K);
                        } else if (keep > cap) {
                            keep = cap;
                        }
                        s_list_count = keep;
                        s_buf_count = 0u;
                    }
                    __syncthreads();
                }
                refresh();
            }

            // ---- change one middle digit: pm = q-adic valuation of u + 1, a -> a2 (both walks)
            if (u + 1 < nblocks) {
                const int mc = s.mchg[u];
                const int pm = mc & 0xff, a = (mc >> 8) & 0xff, a2 = mc >> 16;
                const int sp = B + pm;
#pragma unroll
                for (int w = 0; w < NW; w++) {
                    int* C = Ct + w * kPottsMidTable * kPottsThreads;
                    Ebase[w] += (unsigned)(C[(pm * Q + a2) * kPottsThreads] - C[(pm * Q + a) * kPottsThreads]) +
                                (unsigned)(s.hq[sp * Q + a2] - s.hq[sp * Q + a]);
                    for (int k = 0; k < B; k++) {
                        const int jv = s.Jq[k * n + sp];
                        int* g = Gt + (w * NF + k * Q) * kPottsThreads;
                        // f_k(a) -= J, f_k(a2) += J
                        g[a * kPottsThreads] -= jv;
                        g[a2 * kPottsThreads] += jv;
                    }
                    for (int p2 = 0; p2 < m; p2++) {
                        if (p2 == pm) continue;
                        const int jv = s.Jq[(B + p2) * n + sp];
                        C[(p2 * Q + a) * kPottsThreads] -= jv;
                        C[(p2 * Q + a2) * kPottsThreads] += jv;
                    }
                }
            }
        }
    }
    __syncthreads();
    const int lc = s_list_count;
    for (int i = tid; i < cap; i += blockDim.x) {
        p.list_E[(size_t)blockIdx.x * cap + i] = i < lc ? s.E[i] : kEmptyE;
        p.list_C[(size_t)blockIdx.x * cap + i] = i < lc ? s.C[i] : kEmptyC;
    }
}

size_t potts_walk_smem(int q, int n, int list_cap)
{
    const int B = potts_inner_digits(q);
    return (size_t)2 * list_cap * 12 + (size_t)kPottsWalks * B * q * kPottsThreads * 4 +
           (size_t)kPottsWalks * kPottsMidTable * kPottsThreads * 4 + (size_t)n * n * 4 + (size_t)n * q * 4 +
           (size_t)potts_pow(q, B) * 8 + (size_t)kPottsMaxBlocks * 4;
}

template <int Q>
const void* walk_fn()
{
    return reinterpret_cast<const void*>(&potts_walk_kernel<Q>);
}

// q = 2 runs as an Ising search (bf_low_spectrum_potts maps it); the walk serves q = 3..8
const void* walk_for(int q)
{
    switch (q) {
    case 3: return walk_fn<3>();
    case 4: return walk_fn<4>();
    case 5: return walk_fn<5>();
    case 6: return walk_fn<6>();
    case 7: return walk_fn<7>();
    default: return walk_fn<8>();
    }
}

// ---- FP64 rescoring and direct enumeration -----------------------------------

// Potts energy in FP64 from the caller's J and h, one warp per record
__global__ void __launch_bounds__(256) potts_rescore_kernel(const int* E, const unsigned long long* C, int cap,
                                                            int n, int q, int dtype, const void* J, const void* h,
                                                            double* out)
{
    __shared__ unsigned char dig[8][kMaxN];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < cap; r += nwarps) {
        const bool empty = E[r] == kEmptyE;
        if (!empty && lane == 0) {
            unsigned long long c = C[r];
            for (int i = 0; i < n; i++) {
                dig[wib][i] = (unsigned char)(c % (unsigned long long)q);
                c /= (unsigned long long)q;
            }
        }
        __syncwarp();
        double part = 0.0;
        if (!empty) {
            for (int i = lane; i < n; i += 32) {
                const int di = dig[wib][i];
                double row = load_val(h, dtype, (size_t)i * q + di);
                for (int j = i + 1; j < n; j++)
                    if (dig[wib][j] == di) row += load_val(J, dtype, (size_t)i * n + j);
                part += row;
            }
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) out[r] = empty ? DBL_MAX : part;
        __syncwarp();
    }
}

constexpr int kPottsDirectThreads = 512;

template <typename K>
__global__ void __launch_bounds__(kPottsDirectThreads) potts_direct_kernel(const void* J, const void* h, int n, int q,
                                                                          int dtype, int R, int S, void* energies,
                                                                          unsigned long long* states)
{
    extern __shared__ __align__(16) unsigned char smem[];
    K* key = reinterpret_cast<K*>(smem);
    unsigned long long* cfg = reinterpret_cast<unsigned long long*>(key + R);
    const int space = (int)potts_pow(q, n);
    for (int x = threadIdx.x; x < R; x += blockDim.x) {
        if (x >= space) {
            if constexpr (std::is_same<K, double>::value) key[x] = DBL_MAX;
            else key[x] = LLONG_MAX;
            cfg[x] = kEmptyC;
            continue;
        }
        unsigned char d[kMaxN];
        int y = x;
        for (int i = 0; i < n; i++) {
            d[i] = (unsigned char)(y % q);
            y /= q;
        }
        K e = 0;
        for (int i = 0; i < n; i++) {
            e += (K)load_val(h, dtype, (size_t)i * q + d[i]);
            for (int j = i + 1; j < n; j++)
                if (d[i] == d[j]) e += (K)load_val(J, dtype, (size_t)i * n + j);
        }
        key[x] = e;
        cfg[x] = (unsigned long long)x;
    }
    block_sort(key, cfg, R);
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        static_cast<K*>(energies)[k] = key[k];
        states[k] = cfg[k];
    }
}

__global__ void potts_finalize_int_kernel(const int* E, const unsigned long long* C, int S, const int* qsp,
                                          long long* out, unsigned long long* states)
{
    const int qs = *qsp;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
        out[k] = (long long)(E[k] >> qs);
        states[k] = C[k];
    }
}

__global__ void __launch_bounds__(512) potts_sort_rescored_kernel(const unsigned long long* C, const double* E64,
                                                                  int cap, int S, double* energies,
                                                                  unsigned long long* states)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* cfg = reinterpret_cast<unsigned long long*>(smem);
    double* key = reinterpret_cast<double*>(cfg + cap);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        key[i] = E64[i];
        cfg[i] = C[i];
    }
    block_sort(key, cfg, cap);
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        energies[k] = key[k];
        states[k] = cfg[k];
    }
}

}  // namespace

cudaError_t launch_potts_prep(const void* J, const void* h, int n, int q, int dtype, PottsPrep* prep, WsHeader* hdr,
                              cudaStream_t s)
{
    potts_prep_kernel<<<1, kPottsPrepThreads, 0, s>>>(J, h, n, q, dtype, prep, hdr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_potts_seed(const PottsPrep* prep, int n, int q, unsigned long long space,
                              unsigned long long sample, int per_block, int blocks, int cap, int* outE,
                              unsigned long long* outC, cudaStream_t s)
{
    const size_t smem = (size_t)per_block * 12 + (size_t)n * n * 4 + (size_t)n * q * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(potts_seed_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    potts_seed_kernel<<<blocks, kPottsSeedThreads, smem, s>>>(prep, n, q, space, sample, per_block, cap, outE, outC);
    count_launches(1);
    return cudaGetLastError();
}

int potts_walk_blocks_per_sm(int q, int m, int n, int list_cap)
{
    (void)m;
    if (q < 3 || q > kPottsMaxQ) return 0;
    const void* fn = walk_for(q);
    const size_t smem = potts_walk_smem(q, n, list_cap);
    if (ensure_smem(reinterpret_cast<const void*>(fn), (size_t)(smem)) != cudaSuccess) return 0;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kPottsThreads, smem) != cudaSuccess) return 0;
    return bps;
}

namespace {

// The tables are one per device: a launch waits for the previous Potts walk on the device (an
// event recorded after it) before overwriting them, except inside a stream capture, where that
// event cannot be waited on (a captured search relies on the order of the graph's launches).
constexpr int kPottsMaxDevices = 64;
std::mutex g_ptable_mutex;
cudaEvent_t g_ptable_free[kPottsMaxDevices];

}  // namespace

cudaError_t launch_potts_walk(const PottsParams& p, int grid, cudaStream_t s)
{
    if (p.q < 3 || p.q > kPottsMaxQ) return cudaErrorInvalidValue;
    const size_t smem = potts_walk_smem(p.q, p.n, p.list_cap);
    const void* fn = walk_for(p.q);
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), (size_t)(smem));
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kPottsMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    const bool ordered = cs == cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_ptable_mutex);
    if (ordered) {
        if (!g_ptable_free[dev]) {
            e = cudaEventCreateWithFlags(&g_ptable_free[dev], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        e = cudaStreamWaitEvent(s, g_ptable_free[dev], 0);
        if (e != cudaSuccess) return e;
    }
    const char* prep = reinterpret_cast<const char*>(p.prep);
    e = cudaMemcpyToSymbolAsync(c_pdT, prep + offsetof(PottsPrep, dT), sizeof(c_pdT), 0, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbolAsync(c_pdT16, prep + offsetof(PottsPrep, dT16), sizeof(c_pdT16), 0,
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    switch (p.q) {
    case 3: potts_walk_kernel<3><<<grid, kPottsThreads, smem, s>>>(p); break;
    case 4: potts_walk_kernel<4><<<grid, kPottsThreads, smem, s>>>(p); break;
    case 5: potts_walk_kernel<5><<<grid, kPottsThreads, smem, s>>>(p); break;
    case 6: potts_walk_kernel<6><<<grid, kPottsThreads, smem, s>>>(p); break;
    case 7: potts_walk_kernel<7><<<grid, kPottsThreads, smem, s>>>(p); break;
    default: potts_walk_kernel<8><<<grid, kPottsThreads, smem, s>>>(p); break;
    }
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return ordered ? cudaEventRecord(g_ptable_free[dev], s) : cudaSuccess;
}

cudaError_t launch_potts_direct(const void* J, const void* h, int n, int q, int dtype, int S, void* energies,
                                unsigned long long* states, WsHeader* hdr, cudaStream_t s)
{
    const int space = (int)potts_pow(q, n);
    int R = 1;
    while (R < space) R <<= 1;
    const size_t smem = (size_t)R * 16;
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) return e;
    if (dtype == 0) {
        e = ensure_smem(reinterpret_cast<const void*>(potts_direct_kernel<long long>), (size_t)(smem));
        if (e != cudaSuccess) return e;
        potts_direct_kernel<long long><<<1, kPottsDirectThreads, smem, s>>>(J, h, n, q, dtype, R, S, energies,
                                                                           states);
    } else {
        e = ensure_smem(reinterpret_cast<const void*>(potts_direct_kernel<double>), (size_t)(smem));
        if (e != cudaSuccess) return e;
        potts_direct_kernel<double><<<1, kPottsDirectThreads, smem, s>>>(J, h, n, q, dtype, R, S, energies, states);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_potts_finalize(const int* E, const unsigned long long* C, int cap, int S, int n, int q, int dtype,
                                  const int* qsp, const void* J, const void* h, double* rescore, void* energies,
                                  unsigned long long* states, cudaStream_t s)
{
    if (dtype == 0) {
        potts_finalize_int_kernel<<<(S + 255) / 256, 256, 0, s>>>(E, C, S, qsp, static_cast<long long*>(energies),
                                                                  states);
        count_launches(1);
        return cudaGetLastError();
    }
    potts_rescore_kernel<<<(cap + 7) / 8, 256, 0, s>>>(E, C, cap, n, q, dtype, J, h, rescore);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)cap * 16;
    e = ensure_smem(reinterpret_cast<const void*>(potts_sort_rescored_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    potts_sort_rescored_kernel<<<1, 512, smem, s>>>(C, rescore, cap, S, static_cast<double*>(energies), states);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
