// Preparation (step A0), seed threshold and the direct kernel for tiny
// search spaces.
//
// prep_kernel: one block.  Reads the strict upper triangle of J and h
// (Sec. 2, Eq. (1)), chooses the fixed-point scale 2^q, quantises, bounds the
// rounding residual and builds the tables of the Gray walk.
//
// seed_kernel: evaluates a pseudo-random sample of configurations exactly
// (quantised energies) and leaves one sorted list per block; after the list
// merge, set_tau_kernel stores the S-th lowest sample energy as the first
// threshold.  Any S real configurations bound the S-th lowest energy from
// above, and a random sample of R configurations puts that bound near the
// S / R quantile, so the enumeration starts with few hits.
//
// direct_kernel: one block enumerates all (<= 4096) configurations of the
// search space by the definition, in FP64 (float instances) or int64
// (integer instances), sorts them by (E, c) and writes the S lowest.
#include <cfloat>
#include <climits>
#include <cmath>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

__device__ __forceinline__ double load_value(const void* p, int dtype, size_t idx)
{
    if (dtype == 0) return (double)static_cast<const int*>(p)[idx];
    if (dtype == 1) return (double)static_cast<const float*>(p)[idx];
    return static_cast<const double*>(p)[idx];
}

__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

constexpr int kPrepThreads = 512;

__global__ void __launch_bounds__(kPrepThreads) prep_kernel(const PrepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = p.n;
    double* Jd = reinterpret_cast<double*>(smem);            // n*n (upper triangle used)
    double* hd = Jd + n * n;                                  // n
    double* red = hd + kMaxN;                                 // blockDim
    int* Jq = reinterpret_cast<int*>(red + kPrepThreads);     // kMaxN*kMaxN (row stride n)
    int* hq = Jq + kMaxN * kMaxN;                             // kMaxN
    int* Tq = hq + kMaxN;                                     // 256
    __shared__ int s_q, s_status;
    __shared__ double s_emax, s_delta;

    const int tid = threadIdx.x;
    Prep* out = p.prep;

    // 1. read the strict upper triangle of J and h
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        Jd[idx] = (i < j) ? load_value(p.J, p.dtype, idx) : 0.0;
    }
    for (int i = tid; i < n; i += blockDim.x) hd[i] = load_value(p.h, p.dtype, i);
    __syncthreads();

    // 2. emax = sum_{i<j} |J_ij| + sum_i |h_i| bounds |E| and every local field
    double part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) part += fabs(Jd[idx]);
    for (int i = tid; i < n; i += blockDim.x) part += fabs(hd[i]);
    double emax = block_sum(part, red);

    // 3. scale exponent: emax * 2^q <= 2^29
    if (tid == 0) {
        int status = 0, q = 0;
        if (emax > 0.0) {
            int e;
            frexp(emax, &e);            // emax < 2^e
            q = p.emq_log2 - e;
            if (p.dtype == 0) {
                if (q < 0) status |= kErrRange;  // integer instance too large for int32 fixed point
                if (q > 16) q = 16;              // integers: 16-bit filter lane = 1 energy unit
                if (q < 0) q = 0;
            } else {
                if (q > 200) q = 200;
                if (q < -200) q = -200;
            }
        }
        if (!(emax < 1e300)) status |= kErrRange;  // inf / nan input
        s_q = q;
        s_status = status;
        s_emax = emax;
    }
    __syncthreads();
    const int q = s_q;

    // 4. quantise (symmetric, zero diagonal) and 5. residual bound
    part = 0.0;
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        int a = (i < j) ? i : j, b = (i < j) ? j : i;
        int v = 0;
        if (a != b) {
            double x = Jd[a * n + b];
            double r = rint(ldexp(x, q));
            v = (int)r;
            if (i < j) part += fabs(x - ldexp(r, -q));
        }
        Jq[idx] = v;
    }
    for (int i = tid; i < n; i += blockDim.x) {
        double r = rint(ldexp(hd[i], q));
        hq[i] = (int)r;
        part += fabs(hd[i] - ldexp(r, -q));
    }
    double delta = block_sum(part, red);
    if (tid == 0) s_delta = delta;
    __syncthreads();

    // 6. inner pair energies T[g] = sum_{i<k} J_q,ik s_i s_k over the IB spins walked inside a block
    const int IB = p.inner_bits, IS = 1 << IB;
    for (int g = tid; g < kGrayMaxInnerSteps; g += blockDim.x) {
        int t = 0;
        if (n >= IB && g < IS) {
            for (int i = 0; i < IB; i++) {
                int si = ((g >> i) & 1) ? 1 : -1;
                for (int k = i + 1; k < IB; k++) {
                    int sk = ((g >> k) & 1) ? 1 : -1;
                    t += Jq[i * n + k] * si * sk;
                }
            }
        }
        Tq[g] = t;
    }
    __syncthreads();

    // 8. outputs
    for (int idx = tid; idx < n * n; idx += blockDim.x) out->Jq[idx] = Jq[idx];
    for (int i = tid; i < kMaxN; i += blockDim.x) out->hq[i] = (i < n) ? hq[i] : 0;
    for (int g = tid; g < kGrayMaxInnerSteps; g += blockDim.x) out->T[g] = Tq[g];
    for (int idx = tid; idx < kMaxN * 16; idx += blockDim.x) {
        int j = idx / 16, k = idx % 16;
        int row = (k < IB) ? k : (k < IB + kKeep ? k : -1);
        out->colJ[j][k] = (j < n && row >= 0 && row < n) ? Jq[row * n + j] : 0;
    }
    for (int t = tid; t < kGrayMaxInnerSteps; t += blockDim.x) {
        unsigned v = 0;
        if (t > 0 && t < IS) {
            int g1 = t ^ (t >> 1), g0 = (t - 1) ^ ((t - 1) >> 1);
            int d = (Tq[g1] >> 16) - (Tq[g0] >> 16);     // floor(T / 2^16) differences
            v = (unsigned)d * 65537u;                     // same increment in both 16-bit lanes
        }
        out->L.dT16[t] = v;
    }
    if (tid == 0) {
        int status = s_status;
        if (p.range_flag && *p.range_flag) status |= kErrRange;   // found by the caller's own map
        int W = 0;
        if (p.dtype != 0 && s_delta > 0.0) {
            // candidates must cover 2 delta (quantisation, both directions) plus the FP64
            // evaluation error of the final re-selection, generously bounded.  With
            // delta = 0 every input is a multiple of 2^-q and |E| 2^q <= 2^29, so every
            // FP64 evaluation is exact and the quantised order is the true order (W = 0).
            double eps = 8.0 * (double)n * (double)n * ldexp(1.0, -53) * s_emax;
            double w = ceil(ldexp(2.0 * s_delta + 2.0 * eps, q)) + 2.0;
            if (w > (double)(1 << 28)) { w = (double)(1 << 28); status |= kErrRange; }
            W = (int)w;
        }
        // zero fields: E(c) = E(~c), so the walk covers the configurations with spin n-1 at -1
        // (the lower half of the task range) and the final selection adds the mirrors
        int hz = p.z2_ok;
        for (int i = 0; i < n && hz; i++) hz = hd[i] == 0.0;
        out->L.z2 = hz;
        out->L.status = status;
        out->L.q = q;
        out->L.W = W;
        out->L.tau0 = INT_MAX;
        out->L.delta = s_delta;
        out->L.emax = s_emax;
        p.hdr->tau = INT_MAX;
        p.hdr->status = (unsigned)status;
        p.hdr->task_next = 0ull;
        p.hdr->spill_count = 0u;
    }
}


// ---- seed threshold ----------------------------------------------------

constexpr int kSeedThreads = 512;
// odd multiplier: x -> x * A mod 2^free is a bijection, spreading the sample
constexpr unsigned long long kSeedMul = 0x9E3779B97F4A7C15ull;

__global__ void __launch_bounds__(kSeedThreads) seed_kernel(const Prep* prep, int n, int free_bits,
                                                             unsigned long long hiconst,
                                                             unsigned long long sample, int per_block, int cap,
                                                             int* outE, unsigned long long* outC)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(smem);   // per_block
    int* E = reinterpret_cast<int*>(C + per_block);                        // per_block
    int* Jq = E + per_block;                                               // n*n
    int* hq = Jq + n * n;                                                  // n
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Jq[i] = prep->Jq[i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) hq[i] = prep->hq[i];
    __syncthreads();
    const unsigned long long mask = (free_bits >= 64) ? ~0ull : ((1ull << free_bits) - 1ull);
    const bool full = sample == mask + 1ull;   // whole space sampled: plain enumeration
    for (int k = threadIdx.x; k < per_block; k += blockDim.x) {
        unsigned long long x = (unsigned long long)blockIdx.x * per_block + k;
        if (x >= sample) { E[k] = kEmptyE; C[k] = kEmptyC; continue; }
        unsigned long long c = hiconst | (full ? x : ((x * kSeedMul) & mask));
        int e = 0;
        for (int i = 0; i < n; i++) {
            int row = hq[i];
            const int* Ji = Jq + i * n;
            for (int j = i + 1; j < n; j++) {
                int v = Ji[j];
                row += ((c >> j) & 1ull) ? v : -v;
            }
            e += ((c >> i) & 1ull) ? row : -row;
        }
        E[k] = e;
        C[k] = c;
    }
    block_sort(E, C, per_block);
    for (int i = threadIdx.x; i < cap; i += blockDim.x) {
        outE[(size_t)blockIdx.x * cap + i] = i < per_block ? E[i] : kEmptyE;
        outC[(size_t)blockIdx.x * cap + i] = i < per_block ? C[i] : kEmptyC;
    }
}

__global__ void set_tau_kernel(const int* E, int S, WsHeader* hdr)
{
    hdr->tau = E[S - 1];
    hdr->task_next = 0ull;
    hdr->spill_count = 0u;
}

// ---- direct enumeration of tiny search spaces ------------------------------

constexpr int kDirectThreads = 512;

template <typename K>
__global__ void __launch_bounds__(kDirectThreads) direct_kernel(const void* J, const void* h, int n, int dtype,
                                                                 int S, int free_bits,
                                                                 unsigned long long hiconst, void* energies,
                                                                 unsigned long long* states)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = 1 << free_bits;
    K* key = reinterpret_cast<K*>(smem);
    unsigned long long* cfg = reinterpret_cast<unsigned long long*>(key + R);
    double* Jd = reinterpret_cast<double*>(cfg + R);
    double* hd = Jd + n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        Jd[idx] = (i < j) ? load_value(J, dtype, idx) : 0.0;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) hd[i] = load_value(h, dtype, i);
    __syncthreads();
    for (int x = threadIdx.x; x < R; x += blockDim.x) {
        unsigned long long c = hiconst | (unsigned long long)x;
        K e = 0;
        for (int i = 0; i < n; i++) {
            K si = ((c >> i) & 1ull) ? K(1) : K(-1);
            K row = (K)hd[i];
            for (int j = i + 1; j < n; j++) {
                K v = (K)Jd[i * n + j];
                row += ((c >> j) & 1ull) ? v : -v;
            }
            e += si * row;
        }
        key[x] = e;
        cfg[x] = c;
    }
    block_sort(key, cfg, R);
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        static_cast<K*>(energies)[k] = key[k];
        states[k] = cfg[k];
    }
}

}  // namespace

cudaError_t launch_prep(const PrepParams& p, cudaStream_t s)
{
    size_t smem = (size_t)p.n * p.n * 8 + kMaxN * 8 + kPrepThreads * 8 + kMaxN * kMaxN * 4 + kMaxN * 4 +
                  kGrayMaxInnerSteps * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(prep_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    prep_kernel<<<1, kPrepThreads, smem, s>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seed(const Prep* prep, int n, int free_bits, unsigned long long hiconst,
                        unsigned long long sample, int per_block, int blocks, int cap, int* outE,
                        unsigned long long* outC, cudaStream_t s)
{
    size_t smem = (size_t)per_block * 12 + (size_t)n * n * 4 + kMaxN * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(seed_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    seed_kernel<<<blocks, kSeedThreads, smem, s>>>(prep, n, free_bits, hiconst, sample, per_block, cap, outE, outC);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void tau_min_kernel(WsHeader* hdr, int v) { atomicMin(&hdr->tau, v); }

cudaError_t launch_tau_min(WsHeader* hdr, int v, cudaStream_t s)
{
    tau_min_kernel<<<1, 1, 0, s>>>(hdr, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_tau(const int* E, int S, WsHeader* hdr, cudaStream_t s)
{
    set_tau_kernel<<<1, 1, 0, s>>>(E, S, hdr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_direct(const void* J, const void* h, int n, int dtype, int S, int free_bits,
                          unsigned long long hiconst, void* energies, unsigned long long* states,
                          WsHeader* hdr, cudaStream_t s)
{
    const int R = 1 << free_bits;
    size_t smem = (size_t)R * 16 + (size_t)n * n * 8 + kMaxN * 8 + 64;
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
    if (e != cudaSuccess) return e;
    if (dtype == 0) {
        e = ensure_smem(reinterpret_cast<const void*>(direct_kernel<long long>), (size_t)(smem));
        if (e != cudaSuccess) return e;
        direct_kernel<long long><<<1, kDirectThreads, smem, s>>>(J, h, n, dtype, S, free_bits, hiconst, energies, states);
        count_launches(1);
    } else {
        e = ensure_smem(reinterpret_cast<const void*>(direct_kernel<double>), (size_t)(smem));
        if (e != cudaSuccess) return e;
        direct_kernel<double><<<1, kDirectThreads, smem, s>>>(J, h, n, dtype, S, free_bits, hiconst, energies, states);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace bf
