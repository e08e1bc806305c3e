// Internal definitions shared by the libbf translation units.
//
// Numbers: an instance is screened in exact fixed point.  Couplings and
// fields are scaled by 2^q and rounded to int32 (J_q, h_q) with q chosen so
// that every energy and every local field of the quantised instance stays
// below 2^29 in magnitude; all enumeration arithmetic on the quantised
// instance is then exact in int32.  For integer instances the scaling is
// exact.  For float instances the total rounding residual
//     delta = sum_{i<j} |J_ij - J_q,ij 2^-q| + sum_i |h_i - h_q,i 2^-q|
// bounds |E(c) - E_q(c) 2^-q| for every configuration c, so every member of
// the exact top-S has E_q <= E_q,S + W with W = 2 delta 2^q (+ margin), and
// the final answer is reselected from those candidates after an FP64
// re-evaluation of Eq. (1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bf.h"

namespace bf {

constexpr int kMaxN = 64;
constexpr int kBWalkBits = 9;                    // spins walked inside one unrolled block (batched walker)
constexpr int kBWalkSteps = 1 << kBWalkBits;     // configurations per block and walk (batched walker)
constexpr int kGrayMaxInnerBits = 10;            // the same for the single-instance Gray walk (9 or 10)
constexpr int kGrayMaxInnerSteps = 1 << kGrayMaxInnerBits;
constexpr int kGrayLargeFreeBits = 42;           // searches of >= 2^42 configurations use 10 inner spins

// inner spins of the Gray walk for a search over 2^free_bits configurations: the larger
// block amortises the once-per-block middle flip, the smaller one halves the exact rescans
// of flagged blocks, which dominate short searches
__host__ __device__ constexpr int gray_inner_bits(int free_bits) { return free_bits >= kGrayLargeFreeBits ? 10 : 9; }
constexpr int kKeep = 4;                         // middle spins whose local field is kept in registers
constexpr int kWalks = 4;                        // walks (tasks) per thread: two packed words
constexpr int kGrayThreads = 256;                // block size of the enumeration kernel
constexpr int kSmallFreeBits = 12;               // at most 2^12 configurations: direct kernel
constexpr int kSeedLog2 = 20;                    // at most 2^20 sampled configurations for the seed
constexpr int kDescentMaxBlocks = 256;           // blocks of the local-search seed (one minimum each)
constexpr int kMinListCap = 128;
constexpr int kMaxListCap = 4096;
constexpr int kEmqLog2 = 29;                     // |E_q|, |local field_q| < 2^29

// Device status bits (workspace header).
enum : unsigned {
    kErrSpill = 1u,      // spill area exhausted: records were lost
    kErrWindow = 2u,     // more near-ties than a list can hold
    kErrTimeout = 4u,    // bounded wait gave up
    kErrRange = 8u,      // instance outside the supported fixed-point range
    kErrArg = 16u        // invalid per-instance argument found on the device (batched call)
};

// Workspace header, first 256 bytes of the workspace.
struct alignas(16) WsHeader {
    int tau;                          // smallest known "S-th quantised energy" (upper bound of E_q,S)
    unsigned status;                  // kErr* bits
    unsigned long long task_next;     // dynamic task counter of the enumeration kernel
    unsigned spill_count;             // records written to the spill area
    unsigned pad0;
    unsigned long long total_units;   // batched call: work units in the queue
    unsigned pad[56];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// Per-instance constants produced by the preparation kernel and read on the device by the
// kernels after it (the increments dT16 through a constant table, see GrayParams).
struct PrepLaunch {
    int status;           // kErr* bits found during preparation
    int q;                // fixed-point scale exponent
    int W;                // candidate window in quantised units (0 for integer instances)
    int tau0;             // seed threshold (INT32 max if none)
    double delta;         // quantisation residual bound (energy units)
    double emax;          // sum |J| + sum |h| (energy units)
    int z2;               // 1: zero fields, the walk covers the half space with spin n-1 at -1
    unsigned dT16[kGrayMaxInnerSteps];   // packed 16-bit pair-energy increments of the inner walk
};

struct Prep {
    PrepLaunch L;
    int Jq[kMaxN * kMaxN];        // quantised symmetric couplings, zero diagonal
    int hq[kMaxN];
    int T[kGrayMaxInnerSteps];    // exact inner pair energy T[g] (quantised units)
    int colJ[kMaxN][16];          // column j: J_q[k][j] for the inner spins k, then the kept middle spins
};

// Records: quantised energy (int32) + configuration (uint64), kept in two
// arrays.  Order: (E, c) ascending.
__host__ __device__ inline bool rec_less(int ea, unsigned long long ca, int eb, unsigned long long cb)
{
    return ea < eb || (ea == eb && ca < cb);
}

// splitmix64 finaliser (Steele, Lea, Flood 2014): a bijective 64-bit mix, used to spread
// pseudo-random starting configurations
__host__ __device__ inline unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

constexpr int kEmptyE = 0x7fffffff;
constexpr unsigned long long kEmptyC = ~0ull;

// Workspace layout of bf_low_spectrum.
struct Layout {
    size_t header, prep, listA_E, listA_C, listB_E, listB_C, spill_E, spill_C, rescore, best_E, best_C, total;
    int lists, list_cap;
    unsigned spill_cap;
};

__host__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ inline int next_pow2(int x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__host__ inline int list_capacity(int S)
{
    int c = next_pow2(2 * S);
    if (c < kMinListCap) c = kMinListCap;
    return c;
}

__host__ inline Layout make_layout(int S, int max_blocks, int spill_log2)
{
    Layout L{};
    L.list_cap = list_capacity(S);
    L.lists = max_blocks;
    L.spill_cap = (unsigned)((size_t)1 << spill_log2);
    size_t off = 0;
    L.header = off;   off = align_up(off + sizeof(WsHeader), 256);
    L.prep = off;     off = align_up(off + sizeof(Prep), 256);
    size_t le = (size_t)L.lists * L.list_cap;
    L.listA_E = off;  off = align_up(off + le * 4, 256);
    L.listA_C = off;  off = align_up(off + le * 8, 256);
    size_t lb = (size_t)((L.lists + 1) / 2) * L.list_cap;
    L.listB_E = off;  off = align_up(off + lb * 4, 256);
    L.listB_C = off;  off = align_up(off + lb * 8, 256);
    L.spill_E = off;  off = align_up(off + (size_t)L.spill_cap * 4, 256);
    L.spill_C = off;  off = align_up(off + (size_t)L.spill_cap * 8, 256);
    L.rescore = off;  off = align_up(off + (size_t)L.list_cap * 8, 256);
    L.best_E = off;   off = align_up(off + (size_t)kDescentMaxBlocks * 4, 256);
    L.best_C = off;   off = align_up(off + (size_t)kDescentMaxBlocks * 8, 256);
    L.total = off;
    return L;
}

// ---- kernel parameter blocks -------------------------------------------

// The packed 16-bit pair-energy increments of the unrolled walk (Prep::L.dT16) are read by
// gray_kernel from a __constant__ table that launch_gray fills from the workspace with a
// stream-ordered device-to-device copy; the candidate window W comes from the workspace too,
// so no host synchronisation sits between preparation and enumeration.
struct GrayParams {
    int n, m, nh;                   // spins, walked middle spins, task-index bits
    int free_bits;
    unsigned long long hiconst;     // fixed top bits of every configuration
    unsigned long long ntasks;      // 2^nh
    int S, list_cap, seg_log2;
    unsigned spill_cap;
    int inner_bits;                 // spins of the unrolled block (9 or 10)
    const Prep* prep;
    WsHeader* hdr;
    int* list_E;
    unsigned long long* list_C;
    int* spill_E;
    unsigned long long* spill_C;
};

struct PrepParams {
    const void* J;
    const void* h;
    int n, dtype, S, free_bits;
    unsigned long long hiconst;
    int emq_log2;                   // |E_q| and |local fields| < 2^emq_log2
    int inner_bits;                 // inner spins of the Gray walk the tables are built for
    int z2_ok;                      // the plan allows the half-space walk of zero-field instances
    const unsigned* range_flag;     // optional: nonzero *range_flag marks the instance out of range
    Prep* prep;
    WsHeader* hdr;
};

struct TcParams {                   // tensor-core screening kernel (k_tc.cu); W is read from prep
    int n, m, nh, free_bits;        // m walked outer spins per task, nh task-index bits
    unsigned long long hiconst, ntasks;
    int S, list_cap, seg_log2;
    unsigned spill_cap;
    int delta;                      // widening of the tensor-core test (quantised units)
    int stall_test;                 // testing only: the MMA warps issue nothing (bounded waits run out)
    const Prep* prep;
    WsHeader* hdr;
    int* list_E;
    unsigned long long* list_C;
    int* spill_E;
    unsigned long long* spill_C;
};

// ---- q-state Potts model (k_potts.cu) -----------------------------------

constexpr int kPottsMinQ = 2, kPottsMaxQ = 8;
constexpr int kPottsMaxSteps = 1024;              // configurations of one inner block (q^B)
constexpr int kPottsMidTable = 16;                // max m * q (per-walk middle-digit tables)
constexpr int kPottsMaxBlocks = 256;              // q^m <= 256 blocks per task when m * q <= 16
constexpr int kPottsWalks = 2;                    // walks per thread: two 16-bit lanes of one register

// inner digits walked by the unrolled block for q states (q^B <= kPottsMaxSteps)
__host__ __device__ constexpr int potts_inner_digits(int q)
{
    return q == 2 ? 9 : q == 3 ? 6 : q == 4 ? 5 : q == 5 ? 4 : 3;
}

__host__ __device__ constexpr unsigned long long potts_pow(int q, int e)
{
    unsigned long long r = 1;
    for (int i = 0; i < e; i++) r *= (unsigned long long)q;
    return r;
}

// q-adic valuation of t >= 1 (the digit that changes at step t of the reflected q-ary Gray code)
__host__ __device__ constexpr int potts_qval(unsigned long long t, int q)
{
    int k = 0;
    while (t % (unsigned long long)q == 0ull) { t /= (unsigned long long)q; k++; }
    return k;
}

// digit p of the reflected q-ary Gray code of u
__host__ __device__ constexpr int potts_gray_digit(unsigned long long u, int q, int p)
{
    for (int i = 0; i < p; i++) u /= (unsigned long long)q;
    const int d = (int)(u % (unsigned long long)q);
    return ((u / (unsigned long long)q) & 1ull) ? q - 1 - d : d;
}

struct PottsPrep {                       // written by potts_prep_kernel (device)
    int q, status, qs, W;                // states, status bits, scale exponent, window
    double delta, emax;
    int dT[kPottsMaxSteps];              // inner pair-table difference of Gray step t (t >= 1)
    unsigned dT16[kPottsMaxSteps];       // floor(T / 2^16) differences, same value in both 16-bit lanes
    int Jq[kMaxN * kMaxN];               // quantised symmetric couplings, zero diagonal
    int hq[kMaxN * kPottsMaxQ];          // quantised fields h_i(v), row stride q
};

// The walk reads PottsPrep::dT and ::dT16 from __constant__ tables that launch_potts_walk fills
// from the workspace (device-to-device, stream-ordered) and the window W from the workspace.
struct PottsParams {
    unsigned long long qpow[kMaxN + 1];  // q^i
    int n, q, B, m;                      // spins, states, inner digits, walked middle digits
    unsigned long long ntasks;           // q^(n - B - m)
    int S, list_cap, seg_log2;
    unsigned spill_cap;
    int pad0;
    const PottsPrep* prep;
    WsHeader* hdr;
    int* list_E;
    unsigned long long* list_C;
    int* spill_E;
    unsigned long long* spill_C;
};

cudaError_t launch_potts_prep(const void* J, const void* h, int n, int q, int dtype, PottsPrep* prep,
                              WsHeader* hdr, cudaStream_t s);
cudaError_t launch_potts_seed(const PottsPrep* prep, int n, int q, unsigned long long space,
                              unsigned long long sample, int per_block, int blocks, int cap, int* outE,
                              unsigned long long* outC, cudaStream_t s);
cudaError_t launch_potts_walk(const PottsParams& p, int grid, cudaStream_t s);
int potts_walk_blocks_per_sm(int q, int m, int n, int list_cap);
cudaError_t launch_potts_direct(const void* J, const void* h, int n, int q, int dtype, int S, void* energies,
                                unsigned long long* states, WsHeader* hdr, cudaStream_t s);
// qsp: device, the fixed-point scale exponent (PottsPrep::qs)
cudaError_t launch_potts_finalize(const int* E, const unsigned long long* C, int cap, int S, int n, int q,
                                  int dtype, const int* qsp, const void* J, const void* h, double* rescore,
                                  void* energies, unsigned long long* states, cudaStream_t s);

// ---- batched search ----------------------------------------------------

constexpr int kBMinN = 10;                       // smallest n of the batched walker
constexpr int kBMaxN = 32;                       // largest n of the batched walker
constexpr int kBMaxS = 64;

struct BInst {                                   // per-instance constants (device)
    int n, q, W, m, nh, status;                  // n: spins the walker enumerates
    int n_full, z2;                              // the instance's spins; 1: zero fields, half space walked
    unsigned long long units;                    // work units (128 tasks each)
    double delta, emax;
    int Jq[kBMaxN * kBMaxN];
    int hq[kBMaxN];
    int T[kBWalkSteps];                          // inner pair energies of the walker's block
    unsigned dT16[kBWalkSteps];
    int col[kBMaxN][16];
    // float instances: rounding residuals rho = x - x_q 2^-q as integers round(rho 2^(q+48))
    // (J: strict upper triangle, row stride n; h), for the final re-evaluation of Eq. (1)
    long long R[kBMaxN * kBMaxN];
    long long Rh[kBMaxN];
};
constexpr int kBResBits = 48;                    // fixed-point scale of BInst::R, Rh: 2^(q+48)

struct BatchParams {
    int B, n_max, S, dtype, m_cap, pool_cap, final_len, pad0;
    const void* J;
    const void* h;
    const long long* J_off;
    const long long* h_off;
    const int* n;
    WsHeader* hdr;
    BInst* inst;
    int* tau;
    unsigned* pool_count;
    int* order;
    unsigned long long* wave_off;                // max_waves + 1 entries
    int max_waves, pad1;
    int* pool_E;
    unsigned long long* pool_C;
    void* energies;
    unsigned long long* states;
};

cudaError_t launch_batched(const BatchParams& p, int walker_grid, cudaStream_t s);
cudaError_t launch_backward(const unsigned long long* states, const double* g, const int* n, int B, int S,
                            const long long* J_off, const long long* h_off, void* dJ, void* dh, int out_f64,
                            cudaStream_t s);
int batched_walker_blocks_per_sm();

// ---- launchers (defined in the .cu files) ----------------------------

// Kernels launched by the library (process-wide); every launcher adds its launches.
void count_launches(int k);
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when `bytes` exceeds what was set
// before for this kernel on the current device (the call costs microseconds per launch)
cudaError_t ensure_smem(const void* func, size_t bytes);
// Set the calling thread's error detail (bf_last_error_detail) and return `s`.
bf_status report(bf_status s, const char* detail);

cudaError_t launch_prep(const PrepParams& p, cudaStream_t s);
cudaError_t launch_gray(const GrayParams& p, int grid, cudaStream_t s);
cudaError_t launch_tc(const TcParams& p, int grid, cudaStream_t s);
size_t tc_smem_bytes(int n, int list_cap);
int gray_blocks_per_sm(int list_cap);
size_t gray_smem_bytes(int n, int list_cap);

// Merge of sorted record lists: `nin` lists of `cap` records each in
// (inE, inC) are merged pairwise into ceil(nin / 2) lists in (outE, outC).
// Wp != nullptr: the window is read on the device from *Wp instead of W.
cudaError_t launch_merge_round(const int* inE, const unsigned long long* inC, int nin,
                               int* outE, unsigned long long* outC, int cap, int S, int W,
                               WsHeader* hdr, cudaStream_t s, const int* Wp = nullptr);
// Fold the spill area into the `nlists` lists of (E, C) (grid-stride over chunks).
cudaError_t launch_absorb_spill(int* E, unsigned long long* C, int nlists, int cap, int S, int W,
                                const int* spill_E, const unsigned long long* spill_C,
                                unsigned spill_cap, WsHeader* hdr, cudaStream_t s, const int* Wp = nullptr);
// Small search spaces (k_small.cu): the whole search in one launch of small_search_kernel,
// 2^13 configurations per block (exact Gray enumeration in fixed point), the block lists merged
// up a ticketed tree, the last block writing the S results.  The kernel quantises the instance
// itself (the same rule as the preparation kernel), so nothing else runs before it.
constexpr int kSmallBlockBits = 13;
constexpr int kSmallMaxFreeBits = 20;
struct SmallParams {
    const void* J;                  // caller's n x n couplings (strict upper triangle read)
    const void* h;                  // caller's n fields
    int dtype;                      // 0 int32, 1 float32, 2 float64
    int n, free_bits, S, cap;       // cap: list capacity, 2 cap <= 2^13
    int nlists;                     // blocks = 2^(free_bits - 13)
    unsigned long long hiconst;     // fixed bits of the chunk (Eq. (6))
    const unsigned* range_flag;     // optional: nonzero marks the instance out of range
    int* list_E;                    // nlists lists of cap records (the merge tree's nodes)
    unsigned long long* list_C;
    unsigned* aux;                  // nlists words: status accumulator, then the tree's tickets
    WsHeader* hdr;
    void* energies;                 // S results: int64 (int32 instances) or float64
    unsigned long long* states;
};
int small_lists(int free_bits);
cudaError_t launch_small(const SmallParams& p, cudaStream_t s);

// Final selection: integer instances write E_q >> q; float instances
// re-evaluate Eq. (1) in FP64 from the caller's J, h and reselect.
// qp != nullptr: the scale exponent is read on the device from *qp instead of q.
// z2p != nullptr and *z2p: the list holds the half space with spin n-1 at -1 of a zero-field
// instance; the S outputs include the mirrors c ^ (2^n - 1).
cudaError_t launch_finalize(const int* E, const unsigned long long* C, int cap, int S, int n, int dtype,
                            int q, const void* J, const void* h, double* rescore,
                            void* energies, unsigned long long* states, WsHeader* hdr, cudaStream_t s,
                            const int* qp = nullptr, const int* z2p = nullptr);
// Seed: `blocks` lists of the lowest sampled records (sample configurations in total).
cudaError_t launch_seed(const Prep* prep, int n, int free_bits, unsigned long long hiconst,
                        unsigned long long sample, int per_block, int blocks, int cap, int* outE,
                        unsigned long long* outC, cudaStream_t s);
// Local-search seed (k_descent.cu): `blocks` descent blocks, then the S-th lowest distinct
// energy of the radius-2 Hamming balls around the lowest minima found becomes hdr->tau
// (assign; needs ball_size(free_bits) >= S) or lowers it (atomicMin).
int ball_size(int free_bits);
cudaError_t launch_descent_seed(const Prep* prep, int n, int free_bits, unsigned long long hiconst, int S,
                                int blocks, int* bestE, unsigned long long* bestC, bool assign, WsHeader* hdr,
                                cudaStream_t s);
// hdr->tau = E[S - 1] of a merged list; resets the task and spill counters.
cudaError_t launch_set_tau(const int* E, int S, WsHeader* hdr, cudaStream_t s);
// hdr->tau = min(hdr->tau, v) (v: the quantised energy of S known configurations or more)
cudaError_t launch_tau_min(WsHeader* hdr, int v, cudaStream_t s);
// Small instances (<= 2^kSmallFreeBits configurations): direct enumeration.
// QUBO mapping (k_qubo.cu): dtype 0 = int32 in / int32 out (int64 offset), 1 = float in, 2 = double in
// (double out and offset for both)
cudaError_t launch_qubo_prep(const void* a, const void* b, int n, int dtype, void* Jout, void* hout, void* off4,
                             unsigned* flag, cudaStream_t s);
// map_flag (optional, integer form): nonzero marks the search out of range in *flag (the status word)
cudaError_t launch_qubo_finish(void* F, int S, int dtype, const void* off4, unsigned* flag, cudaStream_t s,
                               const unsigned* map_flag = nullptr);
// Two-state Potts model as an Ising instance (k_qubo.cu): J' = J, h'_i = h_i(1) - h_i(0),
// C = sum_{i<j} J_ij + sum_i (h_i(0) + h_i(1)); energies E = (E' + C) / 2 (same dtypes as the QUBO map)
cudaError_t launch_potts2_prep(const void* J, const void* h, int n, int dtype, void* Jout, void* hout, void* cst,
                               unsigned* flag, cudaStream_t s);
// map_flag (optional, integer form): nonzero marks the search out of range in *flag (the status word)
cudaError_t launch_potts2_finish(void* E, int S, int dtype, const void* cst, unsigned* flag, cudaStream_t s,
                                 const unsigned* map_flag = nullptr);
cudaError_t launch_direct(const void* J, const void* h, int n, int dtype, int S, int free_bits,
                          unsigned long long hiconst, void* energies, unsigned long long* states,
                          WsHeader* hdr, cudaStream_t s);

}  // namespace bf
