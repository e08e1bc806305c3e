// Host side of the C ABI declared in include/bf.h: argument validation,
// launch plan, workspace layout and the kernel sequence of one search.
#include <algorithm>
#include <cstddef>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "bf.h"
#include "bf_internal.cuh"

namespace bf {
static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static std::mutex g_smem_mutex;
static std::map<std::pair<int, const void*>, size_t> g_smem_set;   // (device, kernel) -> bytes allowed

cudaError_t ensure_smem(const void* func, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    size_t& have = g_smem_set[{dev, func}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}
}  // namespace bf

namespace {

thread_local std::string g_detail;

// events of the last profiled call on this host thread
struct ProfileEvents {
    cudaEvent_t start = nullptr, stop = nullptr;
    bool valid = false;
};
thread_local ProfileEvents g_prof;

bf_status fail(bf_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_detail = buf;
    return s;
}

bf_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(BF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ceil_log2(unsigned long long x)
{
    int k = 0;
    while ((1ull << k) < x) k++;
    return k;
}

// autotuned options per (device, n, n - fixed_bits, S, dtype), written by bf_autotune and used
// by make_plan when the caller leaves variant, inner_bits, task_log2 and grid_blocks at 0
using SingleKey = std::tuple<int, int, int, int, int>;
std::mutex g_single_mutex;
std::map<SingleKey, bf_options> g_single_cache;

void apply_single_tune(int n, int S, int dtype, bf_options& o)
{
    if (o.variant || o.inner_bits || o.task_log2 || o.grid_blocks) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(g_single_mutex);
    auto it = g_single_cache.find(SingleKey{dev, n, n - o.fixed_bits, S, dtype});
    if (it == g_single_cache.end()) return;
    o.variant = it->second.variant;
    o.inner_bits = it->second.inner_bits;
    o.task_log2 = it->second.task_log2;
    o.grid_blocks = it->second.grid_blocks;
}

struct Plan {
    int n, S, dtype, free_bits;
    unsigned long long hiconst;
    bool direct;
    int variant;
    int list_cap, grid, m, nh, seg_log2, seed_per_block, seed_blocks, inner_bits;
    int descent_blocks;             // > 0: local-search seed instead of the sampled one
    bool sample_only;               // small space: exact enumeration by k_small.cu, no walk
    unsigned long long seed_sample;
    bf::Layout L;
    size_t bytes;
};

bf_status make_plan(int n, int S, int dtype, const bf_options* opt, Plan& pl)
{
    bf_options o{};
    if (opt) o = *opt;
    apply_single_tune(n, S, dtype, o);
    if (n < 1 || n > bf::kMaxN) return fail(BF_EINVAL, "n=%d outside [1, 64]", n);
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return fail(BF_EINVAL, "unknown dtype %d", dtype);
    if (o.variant != BF_VARIANT_AUTO && o.variant != BF_VARIANT_GRAY && o.variant != BF_VARIANT_TC)
        return fail(BF_EINVAL, "unknown variant %d", o.variant);
    if (o.fixed_bits < 0 || o.fixed_bits > n) return fail(BF_EINVAL, "fixed_bits=%d outside [0, n]", o.fixed_bits);
    const int free_bits = n - o.fixed_bits;
    if (free_bits > 62) return fail(BF_EINVAL, "n - fixed_bits = %d > 62", free_bits);
    if (o.fixed_bits < 64 && o.fixed_bits > 0 && (o.fixed_value >> o.fixed_bits) != 0)
        return fail(BF_EINVAL, "fixed_value does not fit in fixed_bits=%d bits", o.fixed_bits);
    if (o.fixed_bits == 0 && o.fixed_value != 0) return fail(BF_EINVAL, "fixed_value given without fixed_bits");
    if (S < 1) return fail(BF_EINVAL, "S=%d < 1", S);
    if ((unsigned long long)S > (1ull << free_bits)) return fail(BF_EINVAL, "S=%d exceeds 2^%d configurations", S, free_bits);
    if (S > BF_MAX_S) return fail(BF_EUNSUPPORTED, "S=%d exceeds BF_MAX_S=%d", S, BF_MAX_S);
    if (o.task_log2 < 0 || o.grid_blocks < 0) return fail(BF_EINVAL, "negative task_log2 or grid_blocks");
    if (o.spill_log2 < 0 || o.spill_log2 > 28) return fail(BF_EINVAL, "spill_log2=%d outside [0, 28]", o.spill_log2);
    if (o.inner_bits != 0 && o.inner_bits != 9 && o.inner_bits != 10)
        return fail(BF_EINVAL, "inner_bits=%d is not 0, 9 or 10", o.inner_bits);
    // the walk keeps the local fields of the kKeep spins above the inner block
    if (o.inner_bits == 10 && n < 10 + bf::kKeep) return fail(BF_EINVAL, "inner_bits=10 needs n >= 14");

    pl = Plan{};
    pl.n = n;
    pl.S = S;
    pl.dtype = dtype;
    pl.free_bits = free_bits;
    pl.hiconst = o.fixed_bits ? (o.fixed_value << free_bits) : 0ull;
    pl.direct = free_bits <= bf::kSmallFreeBits;
    if (pl.direct) {
        pl.bytes = sizeof(bf::WsHeader);
        return BF_OK;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    pl.list_cap = bf::list_capacity(S);
    pl.variant = o.variant == BF_VARIANT_TC ? BF_VARIANT_TC : BF_VARIANT_GRAY;
    int full_grid = 1;
    if (pl.variant == BF_VARIANT_TC) {
        // one 256-thread block per SM (each holds all 512 TMEM columns); a task is 2^m tiles
        if (free_bits < 15) return fail(BF_EUNSUPPORTED, "the tensor-core variant needs n - fixed_bits >= 15");
        if (bf::tc_smem_bytes(n, pl.list_cap) > (size_t)227 * 1024)
            return fail(BF_EUNSUPPORTED, "S=%d too large for the tensor-core variant", S);
        pl.grid = o.grid_blocks ? o.grid_blocks : sms;
        const int outer = free_bits - 15;
        if (o.task_log2) {
            pl.m = std::min(std::max(o.task_log2 - 15, 0), std::min(outer, 16));
        } else {
            const int tasks = ceil_log2((unsigned long long)pl.grid) + 3;
            pl.m = std::min(std::max(outer - tasks, 0), 16);
        }
        pl.nh = outer - pl.m;
        pl.seg_log2 = std::min(pl.m, 4);
        // a block takes one task at a time: no more blocks than tasks
        full_grid = pl.grid;
        if (!o.grid_blocks && pl.nh < 30) pl.grid = (int)std::min<unsigned long long>(pl.grid, 1ull << pl.nh);
    } else {
        int bps = bf::gray_blocks_per_sm(pl.list_cap);
        if (bps < 1) return fail(BF_ECUDA, "enumeration kernel does not fit on an SM (S=%d)", S);
        pl.grid = o.grid_blocks ? o.grid_blocks : sms * bps;
        pl.inner_bits = o.inner_bits ? o.inner_bits : bf::gray_inner_bits(free_bits);
        const int walk_bits = free_bits - pl.inner_bits;           // middle + task-index bits
        if (o.task_log2) {
            pl.m = std::min(std::max(o.task_log2 - pl.inner_bits, 0), walk_bits);
        } else {
            const int chains = ceil_log2((unsigned long long)pl.grid * bf::kGrayThreads * bf::kWalks);
            pl.m = std::min(std::max(walk_bits - (chains + 2), 0), 14);
        }
        pl.nh = walk_bits - pl.m;
        pl.seg_log2 = std::min(pl.m, 4);
        // a block takes kGrayThreads * kWalks tasks at a time: small searches need fewer blocks,
        // and every block's list goes through the merge tree
        full_grid = pl.grid;
        if (!o.grid_blocks && pl.nh < 40) {
            const unsigned long long per_block = (unsigned long long)bf::kGrayThreads * bf::kWalks;
            const unsigned long long need = ((1ull << pl.nh) + per_block - 1) / per_block;
            pl.grid = (int)std::min<unsigned long long>(pl.grid, need);
        }
    }
    // seed: a pseudo-random sample of up to 2^20 configurations, one sorted list per seed block;
    // sized by the device-filling grid even when the walk needs fewer blocks, so that small
    // searches start from the same threshold quality
    pl.seed_per_block = std::max(pl.list_cap, 2048);
    unsigned long long sample = 1ull << std::min(free_bits, bf::kSeedLog2);
    // spaces of at most 2^20 configurations are enumerated exactly by the small-space kernels
    // (k_small.cu) instead of seed, walk and merges (Gray walk searches with the automatic block
    // size only)
    pl.sample_only = free_bits <= bf::kSmallMaxFreeBits && pl.variant == BF_VARIANT_GRAY && o.inner_bits == 0;
    sample = std::min(sample, (unsigned long long)full_grid * pl.seed_per_block);
    pl.seed_sample = sample;
    pl.seed_blocks = (int)((sample + pl.seed_per_block - 1) / pl.seed_per_block);
    // beyond 2^kSeedLog2 configurations the sample no longer covers the space: a local search
    // and the Hamming balls of its lowest minima give a far lower first threshold (for smaller
    // spaces the sample's exact S-th energy is much tighter than a ball's: a local search
    // threshold at n = 16..24 made the calls 0.26-0.49 ms instead of 0.22-0.26)
    pl.descent_blocks = free_bits > bf::kSeedLog2 ? std::min(sms, bf::kDescentMaxBlocks) : 0;
    int lists = std::max(pl.grid, pl.seed_blocks);
    if (pl.sample_only) lists = std::max(lists, bf::small_lists(free_bits));
    pl.L = bf::make_layout(S, lists, o.spill_log2 ? o.spill_log2 : 21);
    pl.bytes = pl.L.total;
    return BF_OK;
}

// Pairwise merge rounds until one list is left; returns true if it is in A.
cudaError_t merge_tree(int* AE, unsigned long long* AC, int* BE, unsigned long long* BC, int nin, int cap, int S,
                       int W, bf::WsHeader* hdr, cudaStream_t stream, bool& in_a, const int* Wp = nullptr)
{
    in_a = true;
    while (nin > 1) {
        cudaError_t e = in_a ? bf::launch_merge_round(AE, AC, nin, BE, BC, cap, S, W, hdr, stream, Wp)
                             : bf::launch_merge_round(BE, BC, nin, AE, AC, cap, S, W, hdr, stream, Wp);
        if (e != cudaSuccess) return e;
        nin = (nin + 1) / 2;
        in_a = !in_a;
    }
    return cudaSuccess;
}

}  // namespace

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// the converted Ising instance lives after the inner search's workspace
struct QuboLayout {
    size_t inner, J, h, off, flag, total;
};

bf_status qubo_layout(int n, int S, bf_dtype dtype, const bf_options* opt, QuboLayout& q)
{
    const bf_dtype inner_dt = dtype == BF_I32 ? BF_I32 : BF_F64;
    Plan pl;
    bf_status st = make_plan(n, S, inner_dt, opt, pl);
    if (st != BF_OK) return st;
    const size_t elt = dtype == BF_I32 ? 4 : 8;
    q.inner = align256(pl.bytes);
    q.J = q.inner;
    q.h = q.J + align256((size_t)n * n * elt);
    q.off = q.h + align256((size_t)n * elt);
    q.flag = q.off + 8;
    q.total = q.off + 256;
    return BF_OK;
}

}  // namespace

namespace bf {
bf_status report(bf_status s, const char* detail) { return fail(s, "%s", detail); }
}  // namespace bf

namespace {
// tune_configs > 0 (autotuner only): the enumeration kernel takes only the last tasks of its
// queue, about tune_configs configurations; *walked receives their number.  tune_tau: a
// threshold known from an earlier run on the same instance (quantised units), which the walk
// starts from, as the later tasks of a full search do
bf_status low_spectrum_impl(const void* J, const void* h, int n, int S, bf_dtype dtype, void* energies,
                            uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* opt,
                            void* stream_ptr, const unsigned* range_flag, unsigned long long tune_configs = 0,
                            double* walked = nullptr, int tune_tau = 0x7fffffff);
}  // namespace

extern "C" {

size_t bf_workspace_size(int n, int S, bf_dtype dtype, const bf_options* opt)
{
    Plan pl;
    if (make_plan(n, S, dtype, opt, pl) != BF_OK) return 0;
    return pl.bytes;
}

bf_status bf_low_spectrum(const void* J, const void* h, int n, int S, bf_dtype dtype, void* energies,
                          uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* opt,
                          void* stream_ptr)
{
    return low_spectrum_impl(J, h, n, S, dtype, energies, states, workspace, workspace_bytes, opt, stream_ptr,
                             nullptr);
}

}  // extern "C"

namespace {

// range_flag (device, optional): a nonzero value found there when preparation runs marks the
// instance as out of range (the QUBO map's int32 check), without a host round trip
bf_status low_spectrum_impl(const void* J, const void* h, int n, int S, bf_dtype dtype, void* energies,
                            uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* opt,
                            void* stream_ptr, const unsigned* range_flag, unsigned long long tune_configs,
                            double* walked, int tune_tau)
{
    g_detail.clear();
    Plan pl;
    bf_status st = make_plan(n, S, dtype, opt, pl);
    if (st != BF_OK) return st;
    if (walked) *walked = (double)(1ull << pl.free_bits);
    if (!J || !h || !energies || !states || !workspace) return fail(BF_EINVAL, "null pointer argument");
    if (workspace_bytes < pl.bytes)
        return fail(BF_EWORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, pl.bytes);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(BF_EWORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char* ws = static_cast<char*>(workspace);
    auto* hdr = reinterpret_cast<bf::WsHeader*>(ws);
    auto* out_states = reinterpret_cast<unsigned long long*>(states);

    if (pl.direct) {
        cudaError_t e = bf::launch_direct(J, h, n, dtype, S, pl.free_bits, pl.hiconst, energies, out_states, hdr, stream);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "direct kernel");
    }

    const bf::Layout& L = pl.L;
    int* AE = reinterpret_cast<int*>(ws + L.listA_E);
    auto* AC = reinterpret_cast<unsigned long long*>(ws + L.listA_C);
    int* BE = reinterpret_cast<int*>(ws + L.listB_E);
    auto* BC = reinterpret_cast<unsigned long long*>(ws + L.listB_C);
    bool in_a = true;

    if (pl.sample_only) {
        // small space: the whole search in one kernel, 2^13 configurations enumerated exactly per
        // block, the block lists merged up a ticketed tree (k_small.cu); list B holds the tickets
        bf::SmallParams sp{};
        sp.J = J;
        sp.h = h;
        sp.dtype = dtype;
        sp.n = n;
        sp.free_bits = pl.free_bits;
        sp.S = S;
        sp.cap = L.list_cap;
        sp.nlists = bf::small_lists(pl.free_bits);
        sp.hiconst = pl.hiconst;
        sp.range_flag = range_flag;
        sp.list_E = AE;
        sp.list_C = AC;
        sp.aux = reinterpret_cast<unsigned*>(BE);
        sp.hdr = hdr;
        sp.energies = energies;
        sp.states = out_states;
        cudaError_t e = bf::launch_small(sp, stream);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "small-space search");
    }

    auto* prep = reinterpret_cast<bf::Prep*>(ws + L.prep);
    bf::PrepParams pp{};
    pp.J = J;
    pp.h = h;
    pp.n = n;
    pp.dtype = dtype;
    pp.S = S;
    pp.free_bits = pl.free_bits;
    pp.hiconst = pl.hiconst;
    // the tensor-core variant needs 4x headroom: its cross coefficients reach 4 sum|J|
    pp.emq_log2 = pl.variant == BF_VARIANT_TC ? bf::kEmqLog2 - 2 : bf::kEmqLog2;
    pp.inner_bits = pl.variant == BF_VARIANT_TC ? 9 : pl.inner_bits;
    pp.range_flag = range_flag;
    pp.prep = prep;
    pp.hdr = hdr;
    // Zero-field instances walk the half space with spin n-1 at -1 (E(c) = E(~c)); the device
    // decides from h.  Allowed for the Gray walk over the whole space whose first threshold is a
    // single Hamming ball (its distinct configurations map to distinct half-space ones; a sample
    // or a union of balls could hold both c and ~c), when spin n-1 is a task bit (the walk
    // takes the lower half of the task range), and not while the autotuner times a part of the
    // task queue.
    pp.z2_ok = (pl.variant == BF_VARIANT_GRAY && pl.free_bits == n && pl.nh >= 1 && pl.descent_blocks &&
                bf::ball_size(pl.free_bits) >= S && !tune_configs) ? 1 : 0;
    cudaError_t e = bf::launch_prep(pp, stream);
    if (e != cudaSuccess) return cuda_fail(e, "prep kernel");

    const int* Wd = &prep->L.W;
    const int* qd = &prep->L.q;

    // seed threshold: the S-th lowest quantised energy of a pseudo-random sample, and / or of the
    // Hamming balls around local-search minima (alone when the first ball holds S configurations)
    const bool ball_only = pl.descent_blocks && bf::ball_size(pl.free_bits) >= S;
    if (!ball_only) {
        e = bf::launch_seed(prep, n, pl.free_bits, pl.hiconst, pl.seed_sample, pl.seed_per_block, pl.seed_blocks,
                            L.list_cap, AE, AC, stream);
        if (e != cudaSuccess) return cuda_fail(e, "seed kernel");
        e = merge_tree(AE, AC, BE, BC, pl.seed_blocks, L.list_cap, S, 0, hdr, stream, in_a);
        if (e != cudaSuccess) return cuda_fail(e, "seed merge");
        e = bf::launch_set_tau(in_a ? AE : BE, S, hdr, stream);
        if (e != cudaSuccess) return cuda_fail(e, "seed threshold");
    }
    if (pl.descent_blocks) {
        e = bf::launch_descent_seed(prep, n, pl.free_bits, pl.hiconst, S, pl.descent_blocks,
                                    reinterpret_cast<int*>(ws + L.best_E),
                                    reinterpret_cast<unsigned long long*>(ws + L.best_C), ball_only, hdr, stream);
        if (e != cudaSuccess) return cuda_fail(e, "local-search seed");
    }

    // Everything the walk needs from preparation stays on the device: the increments of the
    // unrolled steps go to a constant table (launch_gray), the window W and the scale q are read
    // from the workspace by the kernels, and an instance outside the fixed-point range sets a
    // status bit that stops the walk and is reported by bf_workspace_status.  No host
    // synchronisation: the call can be captured in a CUDA graph.

    bf::GrayParams gp{};
    gp.n = n;
    gp.m = pl.m;
    gp.nh = pl.nh;
    gp.free_bits = pl.free_bits;
    gp.hiconst = pl.hiconst;
    gp.ntasks = 1ull << pl.nh;
    gp.S = S;
    gp.list_cap = L.list_cap;
    gp.seg_log2 = pl.seg_log2;
    gp.inner_bits = pl.inner_bits;
    gp.spill_cap = L.spill_cap;
    gp.prep = prep;
    gp.hdr = hdr;
    gp.list_E = AE;
    gp.list_C = AC;
    gp.spill_E = reinterpret_cast<int*>(ws + L.spill_E);
    gp.spill_C = reinterpret_cast<unsigned long long*>(ws + L.spill_C);
    if (tune_configs) {
        // autotuner: start the task counter near the end of the queue, so that the kernel walks
        // about tune_configs configurations with the full search's task shape
        const int task_bits = (pl.variant == BF_VARIANT_TC ? 15 : pl.inner_bits) + pl.m;
        const unsigned long long ntasks = 1ull << pl.nh;
        const unsigned long long gran = pl.variant == BF_VARIANT_TC ? 1ull : (unsigned long long)bf::kGrayThreads * bf::kWalks;
        // at least two batches of tasks per block, so that every block works as in the full search
        unsigned long long want = std::max((tune_configs >> task_bits) + 1, 2ull * (unsigned long long)pl.grid * gran);
        want = (want + gran - 1) / gran * gran;
        if (want < ntasks) {
            const unsigned long long start = ntasks - want;
            e = cudaMemcpyAsync(&hdr->task_next, &start, sizeof(start), cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "task counter");
            if (walked) *walked = (double)want * (double)(1ull << task_bits);
        }
        if (tune_tau != 0x7fffffff) {
            e = bf::launch_tau_min(hdr, tune_tau, stream);
            if (e != cudaSuccess) return cuda_fail(e, "tuning threshold");
        }
    }
    const bool profile = opt && opt->profile;
    if (profile) {
        if (!g_prof.start) {
            e = cudaEventCreate(&g_prof.start);
            if (e == cudaSuccess) e = cudaEventCreate(&g_prof.stop);
            if (e != cudaSuccess) return cuda_fail(e, "profile events");
        }
        g_prof.valid = false;
        e = cudaEventRecord(g_prof.start, stream);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
    }
    if (pl.variant == BF_VARIANT_TC) {
        bf::TcParams tp{};
        tp.n = n;
        tp.m = pl.m;
        tp.nh = pl.nh;
        tp.free_bits = pl.free_bits;
        tp.hiconst = pl.hiconst;
        tp.ntasks = 1ull << pl.nh;
        tp.S = S;
        tp.list_cap = L.list_cap;
        tp.seg_log2 = pl.seg_log2;
        tp.spill_cap = L.spill_cap;
        // split residuals <= 2^-18 |x| for 8 values below 2^30, FP32 accumulation and conversions
        tp.delta = 1 << 17;
        tp.stall_test = opt ? opt->stall_test : 0;
        tp.prep = prep;
        tp.hdr = hdr;
        tp.list_E = AE;
        tp.list_C = AC;
        tp.spill_E = gp.spill_E;
        tp.spill_C = gp.spill_C;
        e = bf::launch_tc(tp, pl.grid, stream);
    } else {
        e = bf::launch_gray(gp, pl.grid, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "enumeration kernel");
    if (profile) {
        e = cudaEventRecord(g_prof.stop, stream);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
        g_prof.valid = true;
    }

    e = bf::launch_absorb_spill(AE, AC, pl.grid, L.list_cap, S, 0, gp.spill_E, gp.spill_C, L.spill_cap, hdr, stream,
                                Wd);
    if (e != cudaSuccess) return cuda_fail(e, "spill absorb");
    e = merge_tree(AE, AC, BE, BC, pl.grid, L.list_cap, S, 0, hdr, stream, in_a, Wd);
    if (e != cudaSuccess) return cuda_fail(e, "merge rounds");
    const int* FE = in_a ? AE : BE;
    const unsigned long long* FC = in_a ? AC : BC;
    e = bf::launch_finalize(FE, FC, L.list_cap, S, n, dtype, 0, J, h, reinterpret_cast<double*>(ws + L.rescore),
                            energies, out_states, hdr, stream, qd, &prep->L.z2);
    if (e != cudaSuccess) return cuda_fail(e, "finalize");
    return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_workspace_status(const void* workspace, void* stream_ptr)
{
    if (!workspace) return fail(BF_EINVAL, "null workspace");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    unsigned status = 0;
    const auto* hdr = static_cast<const bf::WsHeader*>(workspace);
    cudaError_t e = cudaMemcpyAsync(&status, &hdr->status, sizeof(status), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    if (status & (bf::kErrSpill | bf::kErrWindow))
        return fail(BF_EOVERFLOW, "candidate storage exhausted (device status 0x%x)", status);
    if (status & bf::kErrTimeout) return fail(BF_ETIMEOUT, "bounded device wait expired (device status 0x%x)", status);
    if (status & bf::kErrRange) return fail(BF_EUNSUPPORTED, "instance outside the fixed-point range (0x%x)", status);
    if (status & bf::kErrArg) return fail(BF_EINVAL, "an instance's n is outside the supported range (0x%x)", status);
    return BF_OK;
}

// ---- QUBO form (Sec. 2, Eqs. (2)-(3)) -----------------------------------

size_t bf_qubo_workspace_size(int n, int S, bf_dtype dtype, const bf_options* opt)
{
    QuboLayout q;
    if (qubo_layout(n, S, dtype, opt, q) != BF_OK) return 0;
    return q.total;
}

bf_status bf_low_spectrum_qubo(const void* a, const void* b, int n, int S, bf_dtype dtype, void* F, uint64_t* states,
                               void* workspace, size_t workspace_bytes, const bf_options* opt, void* stream_ptr)
{
    g_detail.clear();
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return fail(BF_EINVAL, "unknown dtype %d", dtype);
    QuboLayout q;
    bf_status st = qubo_layout(n, S, dtype, opt, q);
    if (st != BF_OK) return st;
    if (!a || !b || !F || !states || !workspace) return fail(BF_EINVAL, "null pointer argument");
    if (workspace_bytes < q.total)
        return fail(BF_EWORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, q.total);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(BF_EWORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char* ws = static_cast<char*>(workspace);
    auto* flag = reinterpret_cast<unsigned*>(ws + q.flag);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned), stream);
    if (e == cudaSuccess)
        e = bf::launch_qubo_prep(a, b, n, (int)dtype, ws + q.J, ws + q.h, ws + q.off, flag, stream);
    if (e != cudaSuccess) return cuda_fail(e, "QUBO map");
    // integer inputs whose 2 b_i + sum_j a_ij leaves int32 set the flag; preparation turns it into
    // the out-of-range status (BF_EUNSUPPORTED from bf_workspace_status) and nothing is walked
    const bf_dtype inner_dt = dtype == BF_I32 ? BF_I32 : BF_F64;
    st = low_spectrum_impl(ws + q.J, ws + q.h, n, S, inner_dt, F, states, workspace, q.inner, opt, stream_ptr,
                           flag);
    if (st != BF_OK) return st;
    auto* hdr = reinterpret_cast<bf::WsHeader*>(ws);
    e = bf::launch_qubo_finish(F, S, dtype == BF_I32 ? 0 : 1, ws + q.off, &hdr->status, stream,
                               dtype == BF_I32 ? flag : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "QUBO offset");
    return BF_OK;
}

// ---- q-state Potts model -------------------------------------------------------

namespace {

struct PottsPlan {
    bool direct;
    bool via_ising;                 // q = 2: the Ising search on the mapped instance
    size_t inner, Jp, hp, cst, flag;
    int B, m, grid, seg_log2, list_cap, seed_per_block, seed_blocks;
    unsigned long long space, ntasks, seed_sample;
    bf::Layout L;
    size_t prep_off, bytes;
};

bf_status potts_plan(int n, int q, int S, int dtype, const bf_options* opt, PottsPlan& pl)
{
    bf_options o{};
    if (opt) o = *opt;
    if (q < bf::kPottsMinQ || q > bf::kPottsMaxQ) return fail(BF_EUNSUPPORTED, "q=%d outside [2, 8]", q);
    if (n < 1 || n > bf::kMaxN) return fail(BF_EINVAL, "n=%d outside [1, 64]", n);
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return fail(BF_EINVAL, "unknown dtype %d", dtype);
    if (o.fixed_bits != 0 || o.variant > BF_VARIANT_GRAY) return fail(BF_EINVAL, "fixed_bits / variant not supported for the Potts model");
    unsigned long long space = 1;
    for (int i = 0; i < n; i++) {
        if (space > (1ull << 62) / (unsigned long long)q) return fail(BF_EINVAL, "q^n exceeds 2^62");
        space *= (unsigned long long)q;
    }
    if (S < 1) return fail(BF_EINVAL, "S=%d < 1", S);
    if ((unsigned long long)S > space) return fail(BF_EINVAL, "S=%d exceeds q^n configurations", S);
    if (S > BF_MAX_S) return fail(BF_EUNSUPPORTED, "S=%d exceeds BF_MAX_S=%d", S, BF_MAX_S);
    if (o.spill_log2 < 0 || o.spill_log2 > 28) return fail(BF_EINVAL, "spill_log2=%d outside [0, 28]", o.spill_log2);
    pl = PottsPlan{};
    pl.space = space;
    pl.direct = space <= 4096ull;
    if (pl.direct) {
        pl.bytes = sizeof(bf::WsHeader);
        return BF_OK;
    }
    if (q == 2) {
        // exact reduction to the Ising form: 2 E(sigma) = E'(s) + C with J' = J, h'_i = h_i(1) - h_i(0)
        const bf_dtype inner_dt = dtype == BF_I32 ? BF_I32 : BF_F64;
        Plan ip;
        bf_status st = make_plan(n, S, inner_dt, opt, ip);
        if (st != BF_OK) return st;
        const size_t elt = dtype == BF_I32 ? 4 : 8;
        pl.via_ising = true;
        pl.inner = align256(ip.bytes);
        pl.Jp = pl.inner;
        pl.hp = pl.Jp + align256((size_t)n * n * elt);
        pl.cst = pl.hp + align256((size_t)n * elt);
        pl.flag = pl.cst + 8;
        pl.bytes = pl.cst + 256;
        return BF_OK;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    pl.list_cap = bf::list_capacity(S);
    pl.B = bf::potts_inner_digits(q);
    const int outer = n - pl.B;
    const int bps = bf::potts_walk_blocks_per_sm(q, 0, n, pl.list_cap);
    if (bps < 1) return fail(BF_EUNSUPPORTED, "Potts walk kernel does not fit on an SM (S=%d)", S);
    pl.grid = o.grid_blocks ? o.grid_blocks : sms * bps;
    // enough tasks for ~4 per walk slot, middle digits for the rest (per-thread tables: m q <= 24)
    const unsigned long long want = (unsigned long long)pl.grid * 256ull * bf::kPottsWalks * 4ull;
    int tdig = 0;
    for (unsigned long long c = 1; c < want && tdig < outer; c *= (unsigned long long)q) tdig++;
    int m = outer - tdig;
    m = std::max(0, std::min(m, bf::kPottsMidTable / q));
    pl.m = m;
    pl.ntasks = bf::potts_pow(q, outer - m);
    unsigned long long nb = bf::potts_pow(q, m);
    int lg = 0;
    while ((2ull << lg) <= nb && lg < 4) lg++;
    pl.seg_log2 = lg;
    pl.seed_per_block = std::max(pl.list_cap, 2048);
    unsigned long long sample = std::min(space, 1ull << bf::kSeedLog2);
    sample = std::min(sample, (unsigned long long)pl.grid * pl.seed_per_block);
    pl.seed_sample = sample;
    pl.seed_blocks = (int)((sample + pl.seed_per_block - 1) / pl.seed_per_block);
    pl.L = bf::make_layout(S, pl.grid, o.spill_log2 ? o.spill_log2 : 21);
    pl.prep_off = bf::align_up(pl.L.total, 256);
    pl.bytes = pl.prep_off + bf::align_up(sizeof(bf::PottsPrep), 256);
    return BF_OK;
}

}  // namespace

size_t bf_potts_workspace_size(int n, int q, int S, bf_dtype dtype, const bf_options* opt)
{
    PottsPlan pl;
    if (potts_plan(n, q, S, dtype, opt, pl) != BF_OK) return 0;
    return pl.bytes;
}

bf_status bf_low_spectrum_potts(const void* J, const void* h, int n, int q, int S, bf_dtype dtype, void* energies,
                                uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* opt,
                                void* stream_ptr)
{
    g_detail.clear();
    PottsPlan pl;
    bf_status st = potts_plan(n, q, S, dtype, opt, pl);
    if (st != BF_OK) return st;
    if (!J || !h || !energies || !states || !workspace) return fail(BF_EINVAL, "null pointer argument");
    if (workspace_bytes < pl.bytes)
        return fail(BF_EWORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, pl.bytes);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(BF_EWORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char* ws = static_cast<char*>(workspace);
    auto* hdr = reinterpret_cast<bf::WsHeader*>(ws);
    auto* out_states = reinterpret_cast<unsigned long long*>(states);
    if (pl.direct) {
        cudaError_t e = bf::launch_potts_direct(J, h, n, q, dtype, S, energies, out_states, hdr, stream);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "Potts direct kernel");
    }
    if (pl.via_ising) {
        auto* flag = reinterpret_cast<unsigned*>(ws + pl.flag);
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned), stream);
        if (e == cudaSuccess) e = bf::launch_potts2_prep(J, h, n, (int)dtype, ws + pl.Jp, ws + pl.hp, ws + pl.cst, flag, stream);
        if (e != cudaSuccess) return cuda_fail(e, "two-state Potts map");
        // integer h_i(1) - h_i(0) outside int32 set the flag: preparation turns it into the
        // out-of-range status (BF_EUNSUPPORTED from bf_workspace_status), nothing is walked
        const bf_dtype inner_dt = dtype == BF_I32 ? BF_I32 : BF_F64;
        st = low_spectrum_impl(ws + pl.Jp, ws + pl.hp, n, S, inner_dt, energies, states, workspace, pl.inner, opt,
                               stream_ptr, dtype == BF_I32 ? flag : nullptr);
        if (st != BF_OK) return st;
        e = bf::launch_potts2_finish(energies, S, dtype == BF_I32 ? 0 : 1, ws + pl.cst, &hdr->status, stream,
                                     dtype == BF_I32 ? flag : nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "two-state Potts energies");
        return BF_OK;
    }
    const bf::Layout& L = pl.L;
    auto* prep = reinterpret_cast<bf::PottsPrep*>(ws + pl.prep_off);
    cudaError_t e = bf::launch_potts_prep(J, h, n, q, (int)dtype, prep, hdr, stream);
    if (e != cudaSuccess) return cuda_fail(e, "Potts prep kernel");
    // the walk's constants stay on the device (constant tables filled by launch_potts_walk, the
    // window and scale read from prep by the kernels): no host synchronisation
    const int* Wd = &prep->W;
    const int* qsd = &prep->qs;

    int* AE = reinterpret_cast<int*>(ws + L.listA_E);
    auto* AC = reinterpret_cast<unsigned long long*>(ws + L.listA_C);
    int* BE = reinterpret_cast<int*>(ws + L.listB_E);
    auto* BC = reinterpret_cast<unsigned long long*>(ws + L.listB_C);
    e = bf::launch_potts_seed(prep, n, q, pl.space, pl.seed_sample, pl.seed_per_block, pl.seed_blocks, L.list_cap,
                              AE, AC, stream);
    if (e != cudaSuccess) return cuda_fail(e, "Potts seed kernel");
    bool in_a = true;
    e = merge_tree(AE, AC, BE, BC, pl.seed_blocks, L.list_cap, S, 0, hdr, stream, in_a);
    if (e != cudaSuccess) return cuda_fail(e, "Potts seed merge");
    e = bf::launch_set_tau(in_a ? AE : BE, S, hdr, stream);
    if (e != cudaSuccess) return cuda_fail(e, "Potts seed threshold");

    bf::PottsParams pp{};
    for (int i = 0; i <= bf::kMaxN; i++) pp.qpow[i] = i <= n ? bf::potts_pow(q, i) : 0ull;
    pp.n = n;
    pp.q = q;
    pp.B = pl.B;
    pp.m = pl.m;
    pp.ntasks = pl.ntasks;
    pp.S = S;
    pp.list_cap = L.list_cap;
    pp.seg_log2 = pl.seg_log2;
    pp.spill_cap = L.spill_cap;
    pp.prep = prep;
    pp.hdr = hdr;
    pp.list_E = AE;
    pp.list_C = AC;
    pp.spill_E = reinterpret_cast<int*>(ws + L.spill_E);
    pp.spill_C = reinterpret_cast<unsigned long long*>(ws + L.spill_C);
    const bool profile = opt && opt->profile;
    if (profile) {
        if (!g_prof.start) {
            e = cudaEventCreate(&g_prof.start);
            if (e == cudaSuccess) e = cudaEventCreate(&g_prof.stop);
            if (e != cudaSuccess) return cuda_fail(e, "profile events");
        }
        g_prof.valid = false;
        e = cudaEventRecord(g_prof.start, stream);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
    }
    e = bf::launch_potts_walk(pp, pl.grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "Potts walk kernel");
    if (profile) {
        e = cudaEventRecord(g_prof.stop, stream);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
        g_prof.valid = true;
    }
    e = bf::launch_absorb_spill(AE, AC, pl.grid, L.list_cap, S, 0, pp.spill_E, pp.spill_C, L.spill_cap, hdr, stream,
                                Wd);
    if (e != cudaSuccess) return cuda_fail(e, "spill absorb");
    e = merge_tree(AE, AC, BE, BC, pl.grid, L.list_cap, S, 0, hdr, stream, in_a, Wd);
    if (e != cudaSuccess) return cuda_fail(e, "merge rounds");
    e = bf::launch_potts_finalize(in_a ? AE : BE, in_a ? AC : BC, L.list_cap, S, n, q, (int)dtype, qsd, J, h,
                                  reinterpret_cast<double*>(ws + L.rescore), energies, out_states, stream);
    if (e != cudaSuccess) return cuda_fail(e, "Potts finalize");
    return BF_OK;
}

bf_status bf_last_profile(float* enumeration_ms)
{
    if (!enumeration_ms) return fail(BF_EINVAL, "null output");
    if (!g_prof.valid) return fail(BF_EINVAL, "no profiled call on this thread");
    cudaError_t e = cudaEventSynchronize(g_prof.stop);
    if (e == cudaSuccess) e = cudaEventElapsedTime(enumeration_ms, g_prof.start, g_prof.stop);
    if (e != cudaSuccess) return cuda_fail(e, "profile read");
    return BF_OK;
}

int64_t bf_launch_count(void) { return (int64_t)bf::g_launches.load(std::memory_order_relaxed); }

const char* bf_status_string(bf_status s)
{
    switch (s) {
    case BF_OK: return "BF_OK";
    case BF_EINVAL: return "BF_EINVAL";
    case BF_ECUDA: return "BF_ECUDA";
    case BF_EOVERFLOW: return "BF_EOVERFLOW";
    case BF_ETIMEOUT: return "BF_ETIMEOUT";
    case BF_EUNSUPPORTED: return "BF_EUNSUPPORTED";
    case BF_EWORKSPACE: return "BF_EWORKSPACE";
    }
    return "BF_UNKNOWN";
}

const char* bf_last_error_detail(void) { return g_detail.c_str(); }

const char* bf_version(void) { return "libbf 0.1 (sm_103a)"; }

}  // extern "C"

// ---- batched search ----------------------------------------------------------

namespace {

// autotuned options per (device, B, n_max, S, dtype); used when the caller leaves
// task_log2 and grid_blocks at 0
using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;   // -> (task_log2, grid_blocks)

bf_options effective_batched_options(int B, int n_max, int S, int dtype, const bf_options* opt)
{
    bf_options o{};
    if (opt) o = *opt;
    if (o.task_log2 == 0 && o.grid_blocks == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tune_cache.find(TuneKey{dev, B, n_max, S, dtype});
            if (it != g_tune_cache.end()) {
                o.task_log2 = it->second.first;
                o.grid_blocks = it->second.second;
            }
        }
    }
    return o;
}

struct BPlan {
    int B, n_max, S, dtype, m_cap, pool_cap, final_len, grid, max_waves;
    size_t off_inst, off_tau, off_count, off_order, off_unit, off_poolE, off_poolC, total;
};

bf_status make_bplan(int B, int n_max, int S, int dtype, const bf_options* opt, BPlan& bp)
{
    bf_options o{};
    if (opt) o = *opt;
    if (B < 1) return fail(BF_EINVAL, "B=%d < 1", B);
    if (n_max < bf::kBMinN || n_max > bf::kBMaxN)
        return fail(BF_EUNSUPPORTED, "n_max=%d outside [%d, %d] of the batched search", n_max, bf::kBMinN, bf::kBMaxN);
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return fail(BF_EINVAL, "unknown dtype %d", dtype);
    if (S < 1) return fail(BF_EINVAL, "S=%d < 1", S);
    if (S > bf::kBMaxS) return fail(BF_EUNSUPPORTED, "S=%d exceeds %d for the batched search", S, bf::kBMaxS);
    if (o.task_log2 < 0 || o.grid_blocks < 0) return fail(BF_EINVAL, "negative task_log2 or grid_blocks");
    bp = BPlan{};
    bp.B = B;
    bp.n_max = n_max;
    bp.S = S;
    bp.dtype = dtype;
    // a work unit is 2^10 walks of 2^(kBWalkBits + m) configurations: 2^(kBWalkBits + 10 + m) per unit
    constexpr int kUnitBase = bf::kBWalkBits + 10;
    bp.m_cap = std::min(std::max((o.task_log2 ? o.task_log2 : 25) - kUnitBase, 0), 16);
    const int ubits = std::max(0, n_max - kUnitBase - bp.m_cap);
    const long long units_max = 1ll << ubits;
    long long pool = units_max * S + 512;
    if (pool > 8192) pool = 8192;
    bp.pool_cap = (int)pool;
    bp.final_len = bf::next_pow2(bp.pool_cap);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int bps = bf::batched_walker_blocks_per_sm();
    if (bps < 1) return fail(BF_ECUDA, "batched walker does not fit on an SM");
    bp.grid = o.grid_blocks ? o.grid_blocks : sms * bps;
    size_t off = bf::align_up(sizeof(bf::WsHeader), 256);
    bp.off_inst = off;  off = bf::align_up(off + (size_t)B * sizeof(bf::BInst), 256);
    bp.off_tau = off;   off = bf::align_up(off + (size_t)B * 4, 256);
    bp.off_count = off; off = bf::align_up(off + (size_t)B * 4, 256);
    bp.off_order = off; off = bf::align_up(off + (size_t)B * 4, 256);
    bp.max_waves = (int)units_max;
    bp.off_unit = off;  off = bf::align_up(off + (size_t)(units_max + 1) * 8, 256);
    bp.off_poolE = off; off = bf::align_up(off + (size_t)B * bp.pool_cap * 4, 256);
    bp.off_poolC = off; off = bf::align_up(off + (size_t)B * bp.pool_cap * 8, 256);
    bp.total = off;
    return BF_OK;
}

}  // namespace

extern "C" {

size_t bf_batched_workspace_size(int B, int n_max, int S, bf_dtype dtype, const bf_options* opt)
{
    BPlan bp{};
    const bf_options o = effective_batched_options(B, n_max, S, dtype, opt);
    if (make_bplan(B, n_max, S, dtype, &o, bp) != BF_OK) return 0;
    return bp.total;
}

bf_status bf_low_spectrum_batched(int B, const void* J_packed, const int64_t* J_offsets, const void* h_packed,
                                  const int64_t* h_offsets, const int32_t* n, int n_max, int S, bf_dtype dtype,
                                  void* energies, uint64_t* states, void* workspace, size_t workspace_bytes,
                                  const bf_options* opt, void* stream_ptr)
{
    g_detail.clear();
    BPlan bp{};
    const bf_options eff = effective_batched_options(B, n_max, S, dtype, opt);
    bf_status st = make_bplan(B, n_max, S, dtype, &eff, bp);
    if (st != BF_OK) return st;
    if (!J_packed || !J_offsets || !h_packed || !h_offsets || !n || !energies || !states || !workspace)
        return fail(BF_EINVAL, "null pointer argument");
    if (workspace_bytes < bp.total)
        return fail(BF_EWORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, bp.total);
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(BF_EWORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    char* ws = static_cast<char*>(workspace);
    auto* hdr = reinterpret_cast<bf::WsHeader*>(ws);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(bf::WsHeader), stream);
    if (e != cudaSuccess) return cuda_fail(e, "header reset");
    bf::BatchParams p{};
    p.B = B;
    p.n_max = n_max;
    p.S = S;
    p.dtype = dtype;
    p.m_cap = bp.m_cap;
    p.pool_cap = bp.pool_cap;
    p.final_len = bp.final_len;
    p.J = J_packed;
    p.h = h_packed;
    p.J_off = reinterpret_cast<const long long*>(J_offsets);
    p.h_off = reinterpret_cast<const long long*>(h_offsets);
    p.n = n;
    p.hdr = hdr;
    p.inst = reinterpret_cast<bf::BInst*>(ws + bp.off_inst);
    p.tau = reinterpret_cast<int*>(ws + bp.off_tau);
    p.pool_count = reinterpret_cast<unsigned*>(ws + bp.off_count);
    p.order = reinterpret_cast<int*>(ws + bp.off_order);
    p.wave_off = reinterpret_cast<unsigned long long*>(ws + bp.off_unit);
    p.max_waves = bp.max_waves;
    p.pool_E = reinterpret_cast<int*>(ws + bp.off_poolE);
    p.pool_C = reinterpret_cast<unsigned long long*>(ws + bp.off_poolC);
    p.energies = energies;
    p.states = reinterpret_cast<unsigned long long*>(states);
    e = bf::launch_batched(p, bp.grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched kernels");
    return BF_OK;
}

}  // extern "C"

extern "C" bf_status bf_low_spectrum_backward(const uint64_t* states, const double* grad_E, const int32_t* n, int B,
                                              int S, const int64_t* J_offsets, const int64_t* h_offsets, void* dJ,
                                              void* dh, bf_dtype out_dtype, void* stream_ptr)
{
    g_detail.clear();
    if (B < 1 || S < 1) return fail(BF_EINVAL, "B=%d, S=%d must be >= 1", B, S);
    if (S > 4096) return fail(BF_EUNSUPPORTED, "S=%d exceeds 4096 for the backward kernel", S);
    if (out_dtype != BF_F32 && out_dtype != BF_F64) return fail(BF_EINVAL, "out_dtype must be BF_F32 or BF_F64");
    if (!states || !grad_E || !n || !J_offsets || !h_offsets || !dJ || !dh) return fail(BF_EINVAL, "null pointer argument");
    cudaError_t e = bf::launch_backward(reinterpret_cast<const unsigned long long*>(states), grad_E, n, B, S,
                                        reinterpret_cast<const long long*>(J_offsets),
                                        reinterpret_cast<const long long*>(h_offsets), dJ, dh,
                                        out_dtype == BF_F64 ? 1 : 0, static_cast<cudaStream_t>(stream_ptr));
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "backward kernel");
}

// ---- merge of per-shard results (host) ------------------------------------------

extern "C" bf_status bf_merge_lists(int k, const void* const* energies, const uint64_t* const* states, int S_each,
                                    bf_dtype dtype, int S, void* out_energies, uint64_t* out_states)
{
    g_detail.clear();
    if (k < 1 || S_each < 1 || S < 1) return fail(BF_EINVAL, "k=%d, S_each=%d, S=%d must be >= 1", k, S_each, S);
    if ((long long)k * S_each < S) return fail(BF_EINVAL, "fewer records (%d x %d) than S=%d", k, S_each, S);
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return fail(BF_EINVAL, "unknown dtype %d", dtype);
    if (!energies || !states || !out_energies || !out_states) return fail(BF_EINVAL, "null pointer argument");
    struct Rec { long long ie; double e; uint64_t c; };
    std::vector<Rec> all;
    all.reserve((size_t)k * S_each);
    for (int l = 0; l < k; l++) {
        if (!energies[l] || !states[l]) return fail(BF_EINVAL, "null list %d", l);
        for (int i = 0; i < S_each; i++) {
            Rec r{};
            if (dtype == BF_I32) r.ie = static_cast<const long long*>(energies[l])[i];
            else r.e = static_cast<const double*>(energies[l])[i];
            r.c = states[l][i];
            all.push_back(r);
        }
    }
    const bool is_int = dtype == BF_I32;
    std::sort(all.begin(), all.end(), [is_int](const Rec& a, const Rec& b) {
        if (is_int) { if (a.ie != b.ie) return a.ie < b.ie; }
        else if (a.e != b.e) return a.e < b.e;
        return a.c < b.c;
    });
    // shards cover disjoint subspaces; a configuration listed twice is kept once
    int w = 0;
    for (size_t i = 0; i < all.size() && w < S; i++) {
        if (i > 0 && all[i].c == all[i - 1].c) continue;
        if (is_int) static_cast<long long*>(out_energies)[w] = all[i].ie;
        else static_cast<double*>(out_energies)[w] = all[i].e;
        out_states[w] = all[i].c;
        w++;
    }
    if (w < S) return fail(BF_EINVAL, "only %d distinct records for S=%d", w, S);
    return BF_OK;
}

// ---- autotuner for the single-instance search -------------------------------------

extern "C" bf_status bf_autotune(const void* J, const void* h, int n, int S, bf_dtype dtype, void* energies,
                                 uint64_t* states, void* workspace, size_t workspace_bytes, const bf_options* base,
                                 void* stream_ptr, bf_options* best, double* best_rate, bf_tune_record* records,
                                 int records_cap, int* records_count)
{
    g_detail.clear();
    if (!best) return fail(BF_EINVAL, "null output options");
    if (records_count) *records_count = 0;
    bf_options b0{};
    if (base) b0 = *base;
    b0.variant = 0;
    b0.inner_bits = 0;
    b0.task_log2 = 0;
    b0.grid_blocks = 0;
    b0.profile = 0;
    b0.stall_test = 0;
    Plan pl0;
    {
        bf_options probe = b0;
        probe.variant = BF_VARIANT_GRAY;           // not the cache: validate the arguments as given
        bf_status st = make_plan(n, S, dtype, &probe, pl0);
        if (st != BF_OK) return st;
    }
    if (!J || !h || !energies || !states || !workspace) return fail(BF_EINVAL, "null pointer argument");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");

    // candidates: the Gray walk with 9 and 10 inner spins, the default task length and two
    // either side of it, 1 or 2 blocks per SM; the tensor-core variant where it applies
    std::vector<bf_options> cand;
    if (!pl0.direct && pl0.free_bits <= bf::kSeedLog2) {
        bf_options c = b0;                           // the exact small-space enumeration, no walk
        c.variant = BF_VARIANT_GRAY;
        cand.push_back(c);
    }
    if (!pl0.direct) {
        const int bps = bf::gray_blocks_per_sm(bf::list_capacity(S));
        for (int ib : {9, 10}) {
            if (ib == 10 && n < 10 + bf::kKeep) continue;
            bf_options o = b0;
            o.variant = BF_VARIANT_GRAY;
            o.inner_bits = ib;
            Plan p;
            if (make_plan(n, S, dtype, &o, p) != BF_OK) continue;
            const int walk_bits = pl0.free_bits - ib;
            for (int dm : {0, -2, 2, -4}) {
                const int m = p.m + dm;
                if (dm != 0 && (m < 0 || m > std::min(walk_bits, 14))) continue;
                for (int per_sm = 1; per_sm <= std::max(bps, 1); per_sm++) {
                    bf_options c = o;
                    c.task_log2 = ib + m;
                    c.grid_blocks = sms * per_sm;
                    cand.push_back(c);
                }
            }
        }
        if (pl0.free_bits >= 15) {
            bf_options o = b0;
            o.variant = BF_VARIANT_TC;
            Plan p;
            if (make_plan(n, S, dtype, &o, p) == BF_OK) {
                for (int dm : {0, -2, 2}) {
                    const int m = p.m + dm;
                    if (m < 0 || m > std::min(pl0.free_bits - 15, 16)) continue;
                    bf_options c = o;
                    c.task_log2 = 15 + m;
                    cand.push_back(c);
                }
            }
        }
    } else {
        cand.push_back(b0);                          // tiny space: one kernel, nothing to choose
    }

    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        return fail(BF_ECUDA, "event creation failed");
    // searches beyond 2^39 configurations time the last 2^39 of the task queue
    const unsigned long long tune_configs = pl0.free_bits > 39 ? (1ull << 39) : 0ull;
    double best_r = -1.0;
    bf_options best_o = cand.front();
    int tried = 0;
    int nrec = 0;
    auto note = [&](const bf_options& c, double rate) {
        if (records && nrec < records_cap) {
            records[nrec].opt = c;
            records[nrec].configs_per_s = rate;
            nrec++;
            if (records_count) *records_count = nrec;
        }
    };
    for (const bf_options& c : cand) {
        Plan p;
        if (make_plan(n, S, dtype, &c, p) != BF_OK || p.bytes > workspace_bytes) { note(c, 0.0); continue; }
        double configs = 0.0;
        bf_status st = BF_OK;
        float ms = 0.f;
        int tau_ref = 0x7fffffff;
        for (int rep = 0; rep < 2 && st == BF_OK; rep++) {       // one untimed run, then one timed run
            if (rep == 1 && tune_configs) {
                // the timed part of the queue starts from the threshold the untimed run reached, as
                // the bulk of a full search runs with a threshold close to its final S-th energy
                const auto* hdr = static_cast<const bf::WsHeader*>(workspace);
                e = cudaMemcpyAsync(&tau_ref, &hdr->tau, sizeof(int), cudaMemcpyDeviceToHost, stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
                if (e != cudaSuccess) st = cuda_fail(e, "tuning threshold");
            }
            if (st == BF_OK && rep == 1 && cudaEventRecord(t0, stream) != cudaSuccess) st = fail(BF_ECUDA, "event record");
            if (st == BF_OK)
                st = low_spectrum_impl(J, h, n, S, dtype, energies, states, workspace, workspace_bytes, &c, stream_ptr,
                                       nullptr, tune_configs, &configs, tau_ref);
        }
        if (st == BF_OK) {
            e = cudaEventRecord(t1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess) st = cuda_fail(e, "autotune timing");
        }
        if (st != BF_OK && st != BF_EUNSUPPORTED) {
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            return st;
        }
        if (st != BF_OK) { note(c, 0.0); continue; }
        // a truncated run leaves partial lists: only its time counts.  Device conditions of a
        // full run (overflow) disqualify the candidate.
        if (!tune_configs && bf_workspace_status(workspace, stream_ptr) != BF_OK) { note(c, 0.0); continue; }
        const double rate = configs / (ms * 1e-3);
        note(c, rate);
        tried++;
        if (rate > best_r) { best_r = rate; best_o = c; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (!tried) return fail(BF_EWORKSPACE, "no candidate fits the workspace of %zu bytes", workspace_bytes);
    best_o.fixed_bits = b0.fixed_bits;
    best_o.fixed_value = b0.fixed_value;
    *best = best_o;
    if (best_rate) *best_rate = best_r;
    std::lock_guard<std::mutex> lock(g_single_mutex);
    g_single_cache[SingleKey{dev, n, pl0.free_bits, S, (int)dtype}] = best_o;
    return BF_OK;
}

// ---- autotuner for the batched search ---------------------------------------------

extern "C" bf_status bf_autotune_batched(int B, const void* J_packed, const int64_t* J_offsets, const void* h_packed,
                                         const int64_t* h_offsets, const int32_t* n, int n_max, int S,
                                         bf_dtype dtype, void* energies, uint64_t* states, void* workspace,
                                         size_t workspace_bytes, void* stream_ptr, bf_options* best,
                                         float* best_ms)
{
    g_detail.clear();
    if (!best) return fail(BF_EINVAL, "null output options");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    const int bps = bf::batched_walker_blocks_per_sm();
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        return fail(BF_ECUDA, "event creation failed");
    float best_t = 1e30f;
    bf_options best_o{};
    int tried = 0;
    const int task_candidates[] = {21, 22, 23, 24, 25, 26, 27};
    for (int tl : task_candidates) {
        for (int per_sm = 1; per_sm <= bps; per_sm++) {
            bf_options o{};
            o.task_log2 = tl;
            o.grid_blocks = sms * per_sm;
            BPlan bp{};
            if (make_bplan(B, n_max, S, dtype, &o, bp) != BF_OK) continue;
            if (bp.total > workspace_bytes) continue;       // candidate needs a larger pool
            // one untimed run, then one timed run of the whole batched call
            bf_status st = bf_low_spectrum_batched(B, J_packed, J_offsets, h_packed, h_offsets, n, n_max, S, dtype,
                                                   energies, states, workspace, workspace_bytes, &o, stream);
            if (st != BF_OK) { cudaEventDestroy(t0); cudaEventDestroy(t1); return st; }
            cudaEventRecord(t0, stream);
            st = bf_low_spectrum_batched(B, J_packed, J_offsets, h_packed, h_offsets, n, n_max, S, dtype, energies,
                                         states, workspace, workspace_bytes, &o, stream);
            cudaEventRecord(t1, stream);
            if (st != BF_OK) { cudaEventDestroy(t0); cudaEventDestroy(t1); return st; }
            float ms = 0.f;
            e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e != cudaSuccess) { cudaEventDestroy(t0); cudaEventDestroy(t1); return cuda_fail(e, "autotune timing"); }
            st = bf_workspace_status(workspace, stream);
            if (st != BF_OK) continue;                       // e.g. pool too small for this chunking
            tried++;
            if (ms < best_t) { best_t = ms; best_o = o; }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (!tried) return fail(BF_EWORKSPACE, "no candidate fits the workspace of %zu bytes", workspace_bytes);
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[TuneKey{dev, B, n_max, S, (int)dtype}] = {best_o.task_log2, best_o.grid_blocks};
    return BF_OK;
}
