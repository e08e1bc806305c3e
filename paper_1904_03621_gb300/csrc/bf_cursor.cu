// Resumable exhaustive search (host runtime).
//
// Algorithm 1 (Sec. 3) walks the configuration space in chunks
// c = offset + index (Eq. (6)) and keeps the S lowest records seen so far.
// Here the chunks are the 2^k subspaces whose top k configuration bits equal
// the chunk number; the state between chunks -- the chunk counter and the
// running list of S records -- lives in one caller-owned host buffer, the
// cursor, which can be written to disk and handed back after a restart.
//
// Cursor layout (little-endian, 128-byte header then 2 arrays):
//   header   magic "BFCURSR1", version, n, S, dtype, chunk_bits,
//            next_chunk, total_chunks, instance digest, record count,
//            checksum (FNV-1a 64 of the whole cursor with this field zero)
//   energies S x 8 bytes (int64 for BF_I32, double otherwise), ascending
//   states   S x uint64 configuration integers
#include <algorithm>
#include <cstring>
#include <vector>

#include "bf.h"
#include "bf_internal.cuh"

namespace {

constexpr char kMagic[8] = {'B', 'F', 'C', 'U', 'R', 'S', 'R', '1'};
constexpr uint32_t kVersion = 1;

struct CursorHeader {
    char magic[8];
    uint32_t version;
    int32_t n, S, dtype, chunk_bits, reserved0;
    uint64_t next_chunk, total_chunks;
    uint64_t digest;
    uint64_t count;
    uint64_t checksum;
    uint8_t pad[128 - 8 - 4 - 6 * 4 - 5 * 8];
};
static_assert(sizeof(CursorHeader) == 128, "cursor header size");

constexpr uint64_t kFnvOffset = 1469598103934665603ull, kFnvPrime = 1099511628211ull;

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; i++) {
        h ^= b[i];
        h *= kFnvPrime;
    }
    return h;
}

size_t cursor_bytes(int S) { return sizeof(CursorHeader) + (size_t)16 * (size_t)S; }

uint64_t cursor_checksum(const void* cursor, int S)
{
    CursorHeader h;
    std::memcpy(&h, cursor, sizeof(h));
    h.checksum = 0;
    uint64_t x = fnv1a(kFnvOffset, &h, sizeof(h));
    return fnv1a(x, static_cast<const char*>(cursor) + sizeof(h), (size_t)16 * (size_t)S);
}

size_t elt_size(bf_dtype dt) { return dt == BF_I32 ? 4 : (dt == BF_F32 ? 4 : 8); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// validates a cursor buffer; on success copies its header to *h
bf_status check_cursor(const void* cursor, size_t bytes, CursorHeader* h)
{
    if (!cursor) return bf::report(BF_EINVAL, "null cursor");
    if (bytes < sizeof(CursorHeader)) return bf::report(BF_EINVAL, "cursor buffer shorter than its header");
    std::memcpy(h, cursor, sizeof(*h));
    if (std::memcmp(h->magic, kMagic, 8) != 0) return bf::report(BF_EINVAL, "not a search cursor (bad magic)");
    if (h->version != kVersion) return bf::report(BF_EUNSUPPORTED, "cursor version not supported");
    if (h->S < 1 || h->S > BF_MAX_S || bytes < cursor_bytes(h->S))
        return bf::report(BF_EINVAL, "cursor buffer size does not match its S");
    if (cursor_checksum(cursor, h->S) != h->checksum) return bf::report(BF_EINVAL, "cursor checksum mismatch");
    if (h->next_chunk > h->total_chunks || h->count > (uint64_t)h->S)
        return bf::report(BF_EINVAL, "cursor fields out of range");
    return BF_OK;
}

void seal(void* cursor, CursorHeader& h)
{
    h.checksum = 0;
    std::memcpy(cursor, &h, sizeof(h));
    h.checksum = cursor_checksum(cursor, h.S);
    std::memcpy(cursor, &h, sizeof(h));
}

}  // namespace

extern "C" {

uint64_t bf_instance_digest(const void* J_host, const void* h_host, int n, bf_dtype dtype)
{
    if (!J_host || !h_host || n < 1 || n > 64) return 0;
    const size_t e = elt_size(dtype);
    uint64_t x = fnv1a(kFnvOffset, &n, sizeof(n));
    const int32_t dt = (int32_t)dtype;
    x = fnv1a(x, &dt, sizeof(dt));
    const char* J = static_cast<const char*>(J_host);
    for (int i = 0; i < n; i++)
        x = fnv1a(x, J + ((size_t)i * n + i + 1) * e, (size_t)(n - i - 1) * e);   // strict upper triangle
    return fnv1a(x, h_host, (size_t)n * e);
}

size_t bf_cursor_bytes(int S)
{
    if (S < 1 || S > BF_MAX_S) return 0;
    return cursor_bytes(S);
}

bf_status bf_cursor_init(void* cursor, size_t cursor_bytes_, int n, int S, bf_dtype dtype, int chunk_bits,
                         uint64_t digest)
{
    if (!cursor) return bf::report(BF_EINVAL, "null cursor");
    if (n < 1 || n > 64) return bf::report(BF_EINVAL, "n outside [1, 64]");
    if (dtype != BF_I32 && dtype != BF_F32 && dtype != BF_F64) return bf::report(BF_EINVAL, "unknown dtype");
    if (S < 1 || S > BF_MAX_S) return bf::report(BF_EUNSUPPORTED, "S outside [1, BF_MAX_S]");
    if (chunk_bits < 0 || chunk_bits > n || chunk_bits > 40)
        return bf::report(BF_EINVAL, "chunk_bits outside [0, min(n, 40)]");
    if (n - chunk_bits > 62) return bf::report(BF_EINVAL, "chunks of more than 2^62 configurations");
    if ((unsigned long long)S > (1ull << (n - chunk_bits)))
        return bf::report(BF_EINVAL, "S exceeds the configurations of one chunk");
    if (cursor_bytes_ < cursor_bytes(S)) return bf::report(BF_EINVAL, "cursor buffer too small");
    std::memset(cursor, 0, cursor_bytes(S));
    CursorHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.n = n;
    h.S = S;
    h.dtype = (int32_t)dtype;
    h.chunk_bits = chunk_bits;
    h.next_chunk = 0;
    h.total_chunks = 1ull << chunk_bits;
    h.digest = digest;
    h.count = 0;
    seal(cursor, h);
    return BF_OK;
}

size_t bf_cursor_workspace_size(const void* cursor, size_t cursor_bytes_, const bf_options* opt)
{
    CursorHeader h;
    if (check_cursor(cursor, cursor_bytes_, &h) != BF_OK) return 0;
    bf_options o{};
    if (opt) o = *opt;
    if (o.fixed_bits != 0) return 0;
    o.fixed_bits = h.chunk_bits;
    o.fixed_value = 0;
    const size_t inner = bf_workspace_size(h.n, h.S, (bf_dtype)h.dtype, &o);
    if (inner == 0) return 0;
    return align256(inner) + 2 * align256((size_t)8 * h.S);
}

bf_status bf_cursor_state(const void* cursor, size_t cursor_bytes_, uint64_t* next_chunk, uint64_t* total_chunks,
                          void* energies_host, uint64_t* states_host, int* count)
{
    CursorHeader h;
    bf_status st = check_cursor(cursor, cursor_bytes_, &h);
    if (st != BF_OK) return st;
    if (next_chunk) *next_chunk = h.next_chunk;
    if (total_chunks) *total_chunks = h.total_chunks;
    if (count) *count = (int)h.count;
    const char* body = static_cast<const char*>(cursor) + sizeof(CursorHeader);
    if (energies_host) std::memcpy(energies_host, body, (size_t)8 * h.count);
    if (states_host) std::memcpy(states_host, body + (size_t)8 * h.S, (size_t)8 * h.count);
    return BF_OK;
}

bf_status bf_cursor_step(void* cursor, size_t cursor_bytes_, const void* J, const void* h_dev, int max_chunks,
                         void* workspace, size_t workspace_bytes, const bf_options* opt, void* stream_ptr)
{
    CursorHeader h;
    bf_status st = check_cursor(cursor, cursor_bytes_, &h);
    if (st != BF_OK) return st;
    if (!J || !h_dev || !workspace) return bf::report(BF_EINVAL, "null pointer argument");
    if (max_chunks < 1) return bf::report(BF_EINVAL, "max_chunks < 1");
    if (opt && opt->fixed_bits != 0) return bf::report(BF_EINVAL, "fixed_bits is set by the cursor");
    const size_t need = bf_cursor_workspace_size(cursor, cursor_bytes_, opt);
    if (need == 0) return bf::report(BF_EINVAL, "options rejected for this cursor");
    if (workspace_bytes < need) return bf::report(BF_EWORKSPACE, "workspace smaller than bf_cursor_workspace_size");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return bf::report(BF_EWORKSPACE, "workspace not aligned");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    const int n = h.n, S = h.S;
    const bf_dtype dt = (bf_dtype)h.dtype;

    // the cursor belongs to exactly one instance
    const size_t e = elt_size(dt);
    std::vector<char> Jh((size_t)n * n * e), hh((size_t)n * e);
    cudaError_t ce = cudaMemcpyAsync(Jh.data(), J, Jh.size(), cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hh.data(), h_dev, hh.size(), cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) return bf::report(BF_ECUDA, cudaGetErrorString(ce));
    if (bf_instance_digest(Jh.data(), hh.data(), n, dt) != h.digest)
        return bf::report(BF_EINVAL, "the cursor was made for another instance (digest mismatch)");

    bf_options o{};
    if (opt) o = *opt;
    o.fixed_bits = h.chunk_bits;
    char* ws = static_cast<char*>(workspace);
    const size_t inner = need - 2 * align256((size_t)8 * S);
    void* dE = ws + inner;
    auto* dC = reinterpret_cast<uint64_t*>(ws + inner + align256((size_t)8 * S));
    std::vector<long long> cE_i(S);
    std::vector<double> cE_f(S);
    std::vector<uint64_t> cC(S);
    char* body = static_cast<char*>(cursor) + sizeof(CursorHeader);
    const bool is_int = dt == BF_I32;

    for (int k = 0; k < max_chunks && h.next_chunk < h.total_chunks; k++) {
        o.fixed_value = h.next_chunk;
        st = bf_low_spectrum(J, h_dev, n, S, dt, dE, dC, workspace, inner, &o, stream_ptr);
        if (st != BF_OK) return st;
        st = bf_workspace_status(workspace, stream_ptr);
        if (st != BF_OK) return st;
        ce = cudaMemcpyAsync(is_int ? (void*)cE_i.data() : (void*)cE_f.data(), dE, (size_t)8 * S,
                             cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(cC.data(), dC, (size_t)8 * S, cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) return bf::report(BF_ECUDA, cudaGetErrorString(ce));
        // merge the chunk's S records with the running list (order (E, c) of Algorithm 1)
        struct Rec { long long ie; double e; uint64_t c; };
        std::vector<Rec> all;
        all.reserve((size_t)S + h.count);
        for (uint64_t i = 0; i < h.count; i++) {
            Rec r{};
            std::memcpy(is_int ? (void*)&r.ie : (void*)&r.e, body + 8 * i, 8);
            std::memcpy(&r.c, body + (size_t)8 * S + 8 * i, 8);
            all.push_back(r);
        }
        for (int i = 0; i < S; i++) all.push_back(Rec{is_int ? cE_i[i] : 0, is_int ? 0.0 : cE_f[i], cC[i]});
        std::sort(all.begin(), all.end(), [is_int](const Rec& a, const Rec& b) {
            if (is_int) { if (a.ie != b.ie) return a.ie < b.ie; }
            else if (a.e != b.e) return a.e < b.e;
            return a.c < b.c;
        });
        const size_t keep = std::min(all.size(), (size_t)S);
        for (size_t i = 0; i < keep; i++) {
            std::memcpy(body + 8 * i, is_int ? (const void*)&all[i].ie : (const void*)&all[i].e, 8);
            std::memcpy(body + (size_t)8 * S + 8 * i, &all[i].c, 8);
        }
        h.count = keep;
        h.next_chunk++;
        seal(cursor, h);
    }
    return BF_OK;
}

}  // extern "C"
