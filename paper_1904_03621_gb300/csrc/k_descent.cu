// Local-search seed threshold (part of step A0).
//
// The enumeration prunes with a threshold tau that must bound the S-th lowest
// quantised energy from above; the energy of any S distinct configurations of
// the search space gives such a bound (the S lowest of all configurations are
// at most as high).  The closer tau starts to the true S-th energy, the fewer
// configurations the walk has to record and rescan.
//
// descent_kernel: each warp runs steepest-descent local searches from
// pseudo-random starts on the quantised instance.  Flipping spin i changes the
// energy of Eq. (1) by -2 s_i f_i, with f_i = h_i + sum_j J_ij s_j its local
// field, so the warp repeatedly flips the free spin with the largest s_i f_i > 0
// (a warp maximum over the lanes' spins) and updates all fields
// (f_j += 2 J_ji s_i') until no flip lowers the energy.  Each block writes its
// lowest local minimum (key (E, c)).
//
// ball_kernel: one block takes the lowest distinct minima c* and evaluates
// exactly every configuration within Hamming distance 2 of each over the free
// spins, 1 + f + f(f-1)/2 per centre:
//   E(c* with i flipped)      = E* - 2 s_i f_i
//   E(c* with i, j flipped)   = E* - 2 s_i f_i - 2 s_j f_j + 4 s_i s_j J_ij.
// When the lowest minimum's ball alone holds S configurations, it is the only
// centre and its S-th lowest energy is assigned as the first threshold.
// Otherwise the sampled seed has set a threshold already; the union of the balls
// of up to kBallCenters minima is sorted, repeated records (balls overlap) are
// skipped, and the S-th lowest distinct energy, if the union holds S distinct
// records, lowers the threshold (atomicMin).  The low end of an Ising spectrum
// lies mostly in the few-flip neighbourhoods of its lowest minima, so this bound
// lands far below the S-th energy of a random sample of the same space.
#include <climits>

#include "bf_internal.cuh"
#include "bf_sort.cuh"

namespace bf {
namespace {

constexpr int kDescentThreads = 256;   // eight descents at a time, one per warp
constexpr int kDescentRounds = 4;      // descents per warp
constexpr int kBallThreads = 1024;
constexpr int kBallMax = 4096;        // records of the union of balls (one ball <= 1 + 62 + 62 * 61 / 2)
constexpr int kBallCenters = 8;       // distinct minima whose balls are evaluated
constexpr unsigned long long kDescentSalt = 0x243F6A8885A308D3ull;

// lowest (E, c) of the 32 lanes' records, returned to every lane
__device__ __forceinline__ void warp_min_record(int& e, unsigned long long& c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int e2 = __shfl_xor_sync(0xffffffffu, e, o);
        const unsigned long long c2 = __shfl_xor_sync(0xffffffffu, c, o);
        if (rec_less(e2, c2, e, c)) { e = e2; c = c2; }
    }
}

// One warp per descent: lane l holds the fields of spins l and l + 32.
__global__ void __launch_bounds__(kDescentThreads) descent_kernel(const Prep* prep, int n, int free_bits,
                                                                   unsigned long long hiconst, int* bestE,
                                                                   unsigned long long* bestC)
{
    extern __shared__ __align__(16) int dsm[];
    int* Jq = dsm;                        // n*n (symmetric: column i of row j is J_ij)
    __shared__ int s_E[kDescentThreads / 32];
    __shared__ unsigned long long s_C[kDescentThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n * n; i += kDescentThreads) Jq[i] = prep->Jq[i];
    __syncthreads();

    const int i0 = lane, i1 = lane + 32;
    const bool has0 = i0 < n, has1 = i1 < n;
    const bool free0 = i0 < free_bits, free1 = i1 < free_bits;
    const int h0 = has0 ? prep->hq[i0] : 0, h1 = has1 ? prep->hq[i1] : 0;
    const unsigned long long mask = free_bits >= 64 ? ~0ull : ((1ull << free_bits) - 1ull);
    int bE = kEmptyE;
    unsigned long long bC = kEmptyC;
    for (int r = 0; r < kDescentRounds; r++) {
        const unsigned long long id = ((unsigned long long)blockIdx.x * (kDescentThreads / 32) + warp) * kDescentRounds + r;
        unsigned long long c = hiconst | (splitmix64(kDescentSalt + id) & mask);
        // local fields f_i = h_i + sum_j J_ji s_j (exact modulo 2^32, true values below 2^29)
        unsigned f0 = (unsigned)h0, f1 = (unsigned)h1;
        for (int j = 0; j < n; j++) {
            const bool sj = (c >> j) & 1ull;
            const int* Jj = Jq + j * n;
            if (has0) { const unsigned v = (unsigned)Jj[i0]; f0 += sj ? v : 0u - v; }
            if (has1) { const unsigned v = (unsigned)Jj[i1]; f1 += sj ? v : 0u - v; }
        }
        // 2E = sum_i s_i (f_i + h_i)
        unsigned t = 0u;
        if (has0) { const unsigned fh = f0 + (unsigned)h0; t += ((c >> i0) & 1ull) ? fh : 0u - fh; }
        if (has1) { const unsigned fh = f1 + (unsigned)h1; t += ((c >> i1) & 1ull) ? fh : 0u - fh; }
        int E = (int)__reduce_add_sync(0xffffffffu, t) >> 1;
        // steepest descent: flipping spin i changes E by -2 s_i f_i; every flip lowers E
        for (int it = 0; it < 4 * n; it++) {
            const int v0 = free0 ? ((((c >> i0) & 1ull) ? (int)f0 : -(int)f0)) : INT_MIN;
            const int v1 = free1 ? ((((c >> i1) & 1ull) ? (int)f1 : -(int)f1)) : INT_MIN;
            const int v = v0 >= v1 ? v0 : v1;
            const int best = __reduce_max_sync(0xffffffffu, v);
            if (best <= 0) break;
            const unsigned who = __ballot_sync(0xffffffffu, v == best);
            const int src = __ffs(who) - 1;
            const int k = __shfl_sync(0xffffffffu, v0 >= v1 ? i0 : i1, src);
            c ^= 1ull << k;
            E -= 2 * best;
            const bool up = (c >> k) & 1ull;
            const int* Jk = Jq + k * n;
            if (has0) { const unsigned d = (unsigned)Jk[i0] << 1; f0 += up ? d : 0u - d; }
            if (has1) { const unsigned d = (unsigned)Jk[i1] << 1; f1 += up ? d : 0u - d; }
        }
        if (rec_less(E, c, bE, bC)) { bE = E; bC = c; }
    }
    if (lane == 0) { s_E[warp] = bE; s_C[warp] = bC; }
    __syncthreads();
    if (warp == 0) {
        int e = lane < kDescentThreads / 32 ? s_E[lane] : kEmptyE;
        unsigned long long cc = lane < kDescentThreads / 32 ? s_C[lane] : kEmptyC;
        warp_min_record(e, cc);
        if (lane == 0) { bestE[blockIdx.x] = e; bestC[blockIdx.x] = cc; }
    }
}

__global__ void __launch_bounds__(kBallThreads) ball_kernel(const Prep* prep, int n, int free_bits, int S,
                                                             int nbest, const int* bestE,
                                                             const unsigned long long* bestC, int assign,
                                                             WsHeader* hdr)
{
    extern __shared__ __align__(16) unsigned char bsm[];
    unsigned long long* C = reinterpret_cast<unsigned long long*>(bsm);   // kBallMax
    int* E = reinterpret_cast<int*>(C + kBallMax);                        // kBallMax
    int* Jq = E + kBallMax;                                                // n*n
    __shared__ int s_F[kBallCenters][kMaxN];           // local fields at each centre
    __shared__ int s_cE[kDescentMaxBlocks];
    __shared__ unsigned long long s_cC[kDescentMaxBlocks];
    __shared__ int s_kE[kBallCenters];
    __shared__ unsigned long long s_kC[kBallCenters];
    __shared__ int s_ncent, s_wsum[kBallThreads / 32], s_tau;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n * n; i += kBallThreads) Jq[i] = prep->Jq[i];
    for (int b = tid; b < kDescentMaxBlocks; b += kBallThreads) {
        s_cE[b] = b < nbest ? bestE[b] : kEmptyE;
        s_cC[b] = b < nbest ? bestC[b] : kEmptyC;
    }
    if (tid == 0) s_tau = kEmptyE;
    block_sort(s_cE, s_cC, kDescentMaxBlocks);
    const int f = free_bits;
    const int ball = 1 + f + f * (f - 1) / 2;
    if (warp == 0) {
        // the lowest distinct minima become centres (several blocks may find the same one)
        // one ball when it alone holds S configurations, else the union of up to kBallCenters
        const int kmax = assign ? 1 : min(kBallCenters, kBallMax / ball);
        int k = 0;
        for (int b0 = 0; b0 < kDescentMaxBlocks && k < kmax; b0 += 32) {
            const int b = b0 + lane;
            const bool keep = s_cE[b] != kEmptyE && (b == 0 || s_cE[b] != s_cE[b - 1] || s_cC[b] != s_cC[b - 1]);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int pos = k + __popc(m & ((1u << lane) - 1u));
            if (keep && pos < kmax) { s_kE[pos] = s_cE[b]; s_kC[pos] = s_cC[b]; }
            k += __popc(m);
        }
        if (lane == 0) s_ncent = min(k, kmax);
    }
    __syncthreads();
    const int K = s_ncent;
    for (int x = tid; x < K * kMaxN; x += kBallThreads) {
        const int k = x / kMaxN, i = x % kMaxN;
        if (i >= n) continue;
        const unsigned long long c0 = s_kC[k];
        unsigned fi = (unsigned)prep->hq[i];
        const int* Ji = Jq + i * n;
        for (int j = 0; j < n; j++) {
            const unsigned v = (unsigned)Ji[j];
            fi += ((c0 >> j) & 1ull) ? v : 0u - v;
        }
        s_F[k][i] = (int)fi;
    }
    __syncthreads();
    // slot k * ball + y: centre k; y = 0 the centre, 1..f single flips, then pairs i < j in row order
    const int count = K * ball;
    int len = 1;
    while (len < count) len <<= 1;
    for (int x = tid; x < len; x += kBallThreads) {
        if (x >= count) { E[x] = kEmptyE; C[x] = kEmptyC; continue; }
        const int k = x / ball, y = x % ball;
        const unsigned long long c0 = s_kC[k];
        const int* F = s_F[k];
        unsigned e = (unsigned)s_kE[k];
        unsigned long long cx = c0;
        if (y >= 1 && y <= f) {
            const int i = y - 1;
            const unsigned sf = ((c0 >> i) & 1ull) ? (unsigned)F[i] : 0u - (unsigned)F[i];
            e -= sf << 1;
            cx ^= 1ull << i;
        } else if (y > f) {
            // pair index p -> (i, j): row i holds f - 1 - i pairs
            int p = y - 1 - f, i = 0;
            while (p >= f - 1 - i) { p -= f - 1 - i; i++; }
            const int j = i + 1 + p;
            const bool si = (c0 >> i) & 1ull, sj = (c0 >> j) & 1ull;
            const unsigned fi = si ? (unsigned)F[i] : 0u - (unsigned)F[i];
            const unsigned fj = sj ? (unsigned)F[j] : 0u - (unsigned)F[j];
            const unsigned jij = (unsigned)Jq[i * n + j] << 2;
            e = e - (fi << 1) - (fj << 1) + (si == sj ? jij : 0u - jij);
            cx ^= (1ull << i) | (1ull << j);
        }
        E[x] = (int)e;
        C[x] = cx;
    }
    block_sort(E, C, len);
    // S-th distinct record: balls of different centres overlap, equal records sit side by side
    const int per = (len + kBallThreads - 1) / kBallThreads;
    const int x0 = tid * per;
    int cnt = 0;
    for (int x = x0; x < x0 + per && x < len; x++)
        cnt += E[x] != kEmptyE && (x == 0 || E[x] != E[x - 1] || C[x] != C[x - 1]);
    int incl = cnt;   // inclusive scan over the block
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; w++) before += s_wsum[w];
    int run = before + incl - cnt;   // distinct records before x0
    if (run < S && run + cnt >= S) {
        for (int x = x0; x < x0 + per && x < len; x++) {
            run += E[x] != kEmptyE && (x == 0 || E[x] != E[x - 1] || C[x] != C[x - 1]);
            if (run == S) { s_tau = E[x]; break; }
        }
    }
    __syncthreads();
    if (tid == 0 && s_tau != kEmptyE) {
        if (assign) hdr->tau = s_tau;
        else atomicMin(&hdr->tau, s_tau);
    }
}

}  // namespace

int ball_size(int free_bits) { return 1 + free_bits + free_bits * (free_bits - 1) / 2; }

cudaError_t launch_descent_seed(const Prep* prep, int n, int free_bits, unsigned long long hiconst, int S,
                                int blocks, int* bestE, unsigned long long* bestC, bool assign, WsHeader* hdr,
                                cudaStream_t s)
{
    // assign: the first ball alone holds >= S configurations, so a bound always exists
    if (blocks < 1 || blocks > kDescentMaxBlocks || free_bits > 62 || (assign && ball_size(free_bits) < S))
        return cudaErrorInvalidValue;
    size_t smem = (size_t)n * n * 4;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(descent_kernel), (size_t)(smem));
    if (e != cudaSuccess) return e;
    descent_kernel<<<blocks, kDescentThreads, smem, s>>>(prep, n, free_bits, hiconst, bestE, bestC);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t bsmem = (size_t)kBallMax * 12 + (size_t)n * n * 4;
    e = ensure_smem(reinterpret_cast<const void*>(ball_kernel), (size_t)(bsmem));
    if (e != cudaSuccess) return e;
    ball_kernel<<<1, kBallThreads, bsmem, s>>>(prep, n, free_bits, S, blocks, bestE, bestC, assign ? 1 : 0, hdr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace bf
