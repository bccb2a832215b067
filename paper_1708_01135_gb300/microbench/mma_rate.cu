// Tensor-core instruction rate on this GPU: one thread per SM issues a chain of
// tcgen05.mma kind::f16 (M = 128, K = 16, FP32 accumulation in tensor memory) for several N
// and numbers of independent accumulators, and the clocks per instruction are printed.  It
// is a measurement tool behind the tiling of the reciprocal kernels (recip_tc.cu), not part of
// the library:
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mma_rate mma_rate.cu && ./mma_rate
//
// Operands are constant FP16 ones in shared memory (K-major core-matrix layout, no swizzle);
// every wait is bounded and TMEM is released before exit.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}
__device__ __forceinline__ uint32_t idesc_f16(int M, int N)
{ return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24); }
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__global__ void k(int N, int ndst, int iters, int nB, unsigned long long *out, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x;
    for (int i = t; i < (4096 + 8192 * 4) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(sm)[i] = 0x3c003c00u; // 1.0 halves
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tslot;
    if (t == 0) {
        const uint32_t idesc = idesc_f16(128, N);
        const uint32_t a = su32(sm), b0 = su32(sm + 4096);
        const long long c0 = clock64();
        for (int i = 0; i < iters; ++i) {
            const uint32_t d = tmem + (uint32_t)((i % ndst) * (32 * ((N + 31) / 32)));
            const uint32_t b = b0 + (uint32_t)((i % nB) * 8192);
            umma(d, sdesc(a, 128, 256), sdesc(b, 128, 256), idesc, i >= ndst ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar)) : "memory");
        uint32_t ok = 0;
        long long spins = 0;
        while (!ok && spins < (1ll << 24)) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(ok) : "r"(su32(&bar)), "r"(0u) : "memory");
            ++spins;
        }
        if (!ok) atomicAdd(err, 1);
        const long long c1 = clock64();
        atomicAdd(out, (unsigned long long)(c1 - c0));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}
int main()
{
    unsigned long long *out; int *err;
    cudaMalloc(&out, 8); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
    int nsm = 0; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    const int smem = 4096 + 8192 * 4;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int Ns[] = {64, 96, 128, 144, 208, 256};
    for (int N : Ns)
        for (int ndst : {1, 2, 3})
            for (int nB : {1, 4}) {
                if (ndst * 32 * ((N + 31) / 32) > 512) continue;
                const int iters = 3000;
                cudaMemset(out, 0, 8);
                k<<<nsm, 128, smem>>>(N, ndst, iters, nB, out, err);
                cudaError_t e = cudaDeviceSynchronize();
                unsigned long long cyc = 0; cudaMemcpy(&cyc, out, 8, cudaMemcpyDeviceToHost);
                int er = 0; cudaMemcpy(&er, err, 4, cudaMemcpyDeviceToHost);
                const double per = (double)cyc / nsm / iters;
                printf("N=%3d ndst=%d nB=%d: %7.1f clk/MMA  %7.0f MAC/clk  (%s, timeouts %d)\n", N, ndst, nB, per,
                       128.0 * N * 16 / per, cudaGetErrorString(e), er);
                if (e != cudaSuccess) return 1;
            }
    return 0;
}
