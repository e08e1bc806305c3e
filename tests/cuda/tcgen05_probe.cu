// Self-checking probe of the tcgen05 forms the tensor-core screen relies on (sm_103a):
//   - one tcgen05.mma.cta_group::1.kind::f16, M=128, N=256, K=16, BF16 x BF16 -> F32 in TMEM,
//     operands in shared memory in the no-swizzle K-major layout (leading byte offset 128,
//     stride byte offset 256), committed to an mbarrier;
//   - tcgen05.ld.red.32x32b.x32 .min / .max: the reduction output equals the minimum /
//     maximum of the 32 loaded columns, and the loaded values equal the plain load.
// Exact integer data, so D must match the CPU exactly.  Every wait is bounded; TMEM is
// always freed.  Exit status 0 when everything matches.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

#define LD32(OP, R, MN, A) asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x32." OP ".f32 " \
    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];" \
    : "=r"(R[0]), "=r"(R[1]), "=r"(R[2]), "=r"(R[3]), "=r"(R[4]), "=r"(R[5]), "=r"(R[6]), "=r"(R[7]), \
      "=r"(R[8]), "=r"(R[9]), "=r"(R[10]), "=r"(R[11]), "=r"(R[12]), "=r"(R[13]), "=r"(R[14]), "=r"(R[15]), \
      "=r"(R[16]), "=r"(R[17]), "=r"(R[18]), "=r"(R[19]), "=r"(R[20]), "=r"(R[21]), "=r"(R[22]), "=r"(R[23]), \
      "=r"(R[24]), "=r"(R[25]), "=r"(R[26]), "=r"(R[27]), "=r"(R[28]), "=r"(R[29]), "=r"(R[30]), "=r"(R[31]), "=f"(MN) : "r"(A))

__global__ void __launch_bounds__(128) sem_probe(const uint16_t* A, const uint16_t* B, float* D, float* MN, float* MX,
                                                 unsigned* err)
{
    __shared__ __align__(1024) uint16_t sA[128 * 16];
    __shared__ __align__(1024) uint16_t sB[256 * 16];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int idx = tid; idx < 128 * 16; idx += 128) {
        int r = idx / 16, k = idx % 16;
        sA[((r / 8) * 256 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2) / 2] = A[idx];
    }
    for (int idx = tid; idx < 256 * 16; idx += 128) {
        int r = idx / 16, k = idx % 16;
        sB[((r / 8) * 256 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2) / 2] = B[idx];
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(smem_u32(&tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = tslot;
    if (tid == 0) {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(taddr), "l"(make_desc(smem_u32(sA))), "l"(make_desc(smem_u32(sB))), "r"(idesc), "r"(0));
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&mbar)));
    }
    uint32_t done = 0;
    for (int it = 0; it < 2000000 && !done; it++)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(smem_u32(&mbar)), "r"(0));
    if (!done) atomicOr(err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
        const int row = 32 * warp + lane;
        for (int c = 0; c < 8; c++) {
            uint32_t r[32];
            float mn, mx;
            const uint32_t a = taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c);
            LD32("min", r, mn, a);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            for (int j = 0; j < 32; j++) D[row * 256 + 32 * c + j] = __uint_as_float(r[j]);
            MN[row * 8 + c] = mn;
            uint32_t r2[32];
            LD32("max", r2, mx, a);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            MX[row * 8 + c] = mx;
            for (int j = 0; j < 32; j++) if (r2[j] != r[j]) atomicOr(err, 2u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(taddr));
}

static uint16_t bf16_of_int(int v) { float f = (float)v; uint32_t u; memcpy(&u, &f, 4); return (uint16_t)(u >> 16); }

int main()
{
    uint16_t hA[128 * 16], hB[256 * 16];
    int iA[128 * 16], iB[256 * 16];
    srand(11);
    for (int i = 0; i < 128 * 16; i++) { iA[i] = (rand() % 3) - 1; hA[i] = bf16_of_int(iA[i]); }
    for (int i = 0; i < 256 * 16; i++) { iB[i] = (rand() % 201) - 100; hB[i] = bf16_of_int(iB[i]); }
    uint16_t *dA, *dB;
    float *dD, *dMN, *dMX;
    unsigned* dErr;
    cudaMalloc(&dA, sizeof(hA));
    cudaMalloc(&dB, sizeof(hB));
    cudaMalloc(&dD, 128 * 256 * 4);
    cudaMalloc(&dMN, 128 * 8 * 4);
    cudaMalloc(&dMX, 128 * 8 * 4);
    cudaMalloc(&dErr, 4);
    cudaMemcpy(dA, hA, sizeof(hA), cudaMemcpyHostToDevice);
    cudaMemcpy(dB, hB, sizeof(hB), cudaMemcpyHostToDevice);
    cudaMemset(dErr, 0, 4);
    sem_probe<<<1, 128>>>(dA, dB, dD, dMN, dMX, dErr);
    cudaError_t e = cudaDeviceSynchronize();
    static float hD[128 * 256], hMN[128 * 8], hMX[128 * 8];
    unsigned herr = 0;
    cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(hD, dD, sizeof(hD), cudaMemcpyDeviceToHost);
    cudaMemcpy(hMN, dMN, sizeof(hMN), cudaMemcpyDeviceToHost);
    cudaMemcpy(hMX, dMX, sizeof(hMX), cudaMemcpyDeviceToHost);
    long bad = 0, badmn = 0, badmx = 0;
    for (int m = 0; m < 128; m++) {
        for (int n = 0; n < 256; n++) {
            int ref = 0;
            for (int k = 0; k < 16; k++) ref += iA[m * 16 + k] * iB[n * 16 + k];
            if (hD[m * 256 + n] != (float)ref) bad++;
        }
        for (int c = 0; c < 8; c++) {
            float mn = 1e30f, mx = -1e30f;
            for (int j = 0; j < 32; j++) { float v = hD[m * 256 + 32 * c + j]; mn = v < mn ? v : mn; mx = v > mx ? v : mx; }
            if (hMN[m * 8 + c] != mn) badmn++;
            if (hMX[m * 8 + c] != mx) badmx++;
        }
    }
    printf("semantics: cuda=%s err=%u D mismatches=%ld  min mismatches=%ld  max mismatches=%ld (of %d)  mn[0]=%g mx[0]=%g\n",
           cudaGetErrorString(e), herr, bad, badmn, badmx, 128 * 8, hMN[0], hMX[0]);
    if (e != cudaSuccess) return 1;
    return (herr == 0 && bad == 0 && badmn == 0 && badmx == 0) ? 0 : 2;
}
