// Reciprocal-space sum on the tcgen05 tensor cores (hot-path steps a5-a8, EWALD_MIXED and
// EWALD_MIXED_BF16).
//
// The two matrix-vector products of Eq. 3 (Algorithm 1: rho_hat_k from all particles;
// Algorithm 2: forces from all k) are evaluated as real matrix products on the tensor cores,
// with the k vectors grouped in rows r = (m_y, m_z) and m_x along the row (the row/column
// algebra, including the pairing of +m_x with -m_x, is documented in recip_simt.cu):
//
//   forward  (a6):  D_f[(Re|Im) A[r], col] = sum_j A_j[r] X_j[col]
//                   A_j[r] = q_j e^{i(k_y y_j + k_z z_j)},  cols: Re X_j[m], m = 0..k_max,
//                   then Im X_j[m], m = 1..k_max;  M = 2R, N = 2 k_max + 1, K = particles
//   back     (a8):  D_b[i, col] = sum_r (Re P_i[r], Im P_i[r]) . G'[(r, re|im), col]
//                   P_i[r] = e^{i(k_y y_i + k_z z_i)};  M = particles, N = 3 (2 k_max + 1),
//                   K = 2R
//
// Operands are produced in shared memory, not read from HBM: phase factors come from exact
// 32-bit fixed-point angles (m_y u_y + m_z u_z mod 2^32, u = x / L in units of 2^-32) and
// one sincos each.  Every FP32 operand value v is split into two half-precision terms
// hi = rn(v), lo = rn(v - hi); each product uses hi*hi + hi*lo + lo*hi, accumulated in FP32
// in tensor memory (TMEM).  The back-scatter coefficient matrix G' is scaled by a power of
// two before the FP16 split so that its largest entry sits near 2^14 (FP16 range); the
// epilogue removes the scale.
//
// Kernel structure (one CTA per tile, warp-specialised, mbarrier pipeline in shared memory):
//   warps 0-3  produce the generated operand of each stage, then run the epilogue (warp w
//              owns TMEM lanes 32w..32w+31, i.e. rows of the accumulator)
//   warp 4     (back-scatter) streams the pre-packed G' tiles with bulk TMA copies
//   warp 5     (warp 4 in the forward kernel) issues tcgen05.mma from one thread and
//              releases stages with tcgen05.commit
// Shared-memory operand layout (no swizzle, K-major): 8x8 core matrices of 128 contiguous
// bytes, ordered [row / 8][k / 8][row % 8][k % 8]; descriptor LBO = 128 B (next core matrix
// along K), SBO = (K_stage / 8) * 128 B (next 8-row group).
// Every mbarrier wait is bounded (~1 s of globaltimer); a timeout sets a status bit and
// lets every role leave its loop; the MMA thread's final commit is always issued and
// waited for before TMEM is released.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace ew {
namespace {

// ---- tiling ---------------------------------------------------------------------------
constexpr int kFK = 64;        // forward: particles (K) per stage
constexpr int kFStages = 2;
constexpr int kFMT = 2;        // forward: M tiles (64 rows r = 128 matrix rows) per CTA
constexpr int kFThreads = 160;
constexpr int kBK = 32;        // back-scatter: real K per stage (16 rows r)
constexpr int kBStages = 3;
constexpr int kBMT = 2;        // back-scatter: M tiles of 128 particles per CTA
constexpr int kBThreads = 192;
constexpr int kPassMax = 256;  // N columns per back-scatter pass (one MMA)

// ---- PTX wrappers -----------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(uint64_t *b, uint32_t c)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mb_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mb_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mb_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su32(b)), "r"(parity) : "memory");
    return ok;
}
__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar)) : "memory");
}

constexpr uint64_t kWaitNs = 1000000000ull;

// One-thread bounded wait; false on timeout (sets *abort) or when another role aborted.
__device__ __forceinline__ bool wait1(uint64_t *b, uint32_t parity, volatile int *abort)
{
    const uint64_t t0 = gtime();
    while (!mb_try(b, parity)) {
        if (*abort) return false;
        if (gtime() - t0 > kWaitNs) { *abort = 1; return false; }
    }
    return true;
}

// Whole-warp bounded wait.
__device__ __forceinline__ bool waitw(uint64_t *b, uint32_t parity, volatile int *abort)
{
    const uint64_t t0 = gtime();
    while (true) {
        const uint32_t ok = mb_try(b, parity);
        if (__all_sync(0xffffffffu, ok)) return true;
        const bool stop = *abort || (gtime() - t0 > kWaitNs);
        if (__any_sync(0xffffffffu, stop)) {
            *abort = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void tm_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices, Blackwell version bit.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = FP32, A = B = FP16 (0) or BF16 (1), both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Split a pair of FP32 values into packed hi and lo half-precision pairs.
template <bool BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    if (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        float2 f = __bfloat1622float2(h);
        __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = *reinterpret_cast<uint32_t *>(&l);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        float2 f = __half22float2(h);
        __half2 l = __floats2half2_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<uint32_t *>(&h);
        lo = *reinterpret_cast<uint32_t *>(&l);
    }
}

// e^{2 pi i a / 2^32} for a 32-bit fixed-point angle a (turns).
__device__ __forceinline__ void phase(uint32_t a, float &c, float &s)
{
    const float t = (float)(int32_t)a * 1.4629180792671596e-9f;   // 2 pi / 2^32
    __sincosf(t, &s, &c);
}

// Byte offset of the 16-byte chunk (row, kchunk) in a [row/8][k/8][8][8] tile of
// `kchunks` K-chunks.
__device__ __forceinline__ uint32_t tile_off(int row, int kc, int kchunks)
{
    return (uint32_t)(((row >> 3) * kchunks + kc) * 128 + (row & 7) * 16);
}

__device__ __forceinline__ void st16(unsigned char *base, uint32_t off, uint32_t a, uint32_t b,
                                     uint32_t c, uint32_t d)
{
    *reinterpret_cast<uint4 *>(base + off) = make_uint4(a, b, c, d);
}

// ---- forward: structure-factor partials ------------------------------------------------
// grid (M groups of kFMT tiles, K splits); block kFThreads.
// spart layout [ks][R][k_max + 1][4] = (T_rr, T_ri, T_ir, T_ii), FP32.
template <bool BF>
__global__ void __launch_bounds__(kFThreads, 1)
k_fwd_tc(int n, int R, int kmax, int NF, int per, const RowInfo *__restrict__ rows,
         const uint4 *__restrict__ pu, float *__restrict__ spart, int *__restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int A_BYTES = 128 * kFK * 2;
    const int B_BYTES = NF * kFK * 2;
    const int STAGE = kFMT * 2 * A_BYTES + 2 * B_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + kFStages * STAGE);
    uint64_t *empty = full + kFStages;
    uint64_t *accf = empty + kFStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int mgroup = blockIdx.x, ks = blockIdx.y;
    const int p0 = ks * per;
    const int p1 = min(n, p0 + per);
    const int nst = (p1 - p0 + kFK - 1) / kFK;
    const int kchunks = kFK / 8;

    if (t == 0) {
        for (int s = 0; s < kFStages; ++s) { mb_init(&full[s], 128); mb_init(&empty[s], 1); }
        mb_init(accf, 1);
        *abort = 0;
        mb_fence_init();
    }
    if (warp == 0) { tm_alloc(tslot, 256); tm_relinquish(); }
    // zero the padding columns of B once (no stage writes them)
    for (int u = t; u < kFStages * 2 * (NF - (2 * kmax + 1)) * kchunks; u += kFThreads) {
        int kc = u % kchunks, rest = u / kchunks;
        int col = 2 * kmax + 1 + rest % (NF - (2 * kmax + 1));
        int sp = rest / (NF - (2 * kmax + 1));    // stage * 2 + part
        unsigned char *bt = sm + (sp >> 1) * STAGE + kFMT * 2 * A_BYTES + (sp & 1) * B_BYTES;
        st16(bt, tile_off(col, kc, kchunks), 0u, 0u, 0u, 0u);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    if (t < 128) {
        // ---- producers ----
        for (int it = 0; it < nst; ++it) {
            const int s = it % kFStages, u = it / kFStages;
            if (u > 0 && !waitw(&empty[s], (u - 1) & 1, abort)) break;
            unsigned char *st = sm + s * STAGE;
            const int j0 = p0 + it * kFK;
            // A: (row r', particle chunk c), rows [0, 64) real parts, [64, 128) imaginary
#pragma unroll 1
            for (int mt = 0; mt < kFMT; ++mt) {
                unsigned char *ahi = st + (mt * 2 + 0) * A_BYTES;
                unsigned char *alo = st + (mt * 2 + 1) * A_BYTES;
#pragma unroll 1
                for (int v = 0; v < 4; ++v) {
                    const int unit = t + 128 * v;
                    const int rl = unit & 63, c = unit >> 6;
                    const int gr = (mgroup * kFMT + mt) * 64 + rl;
                    float re[8], im[8];
                    if (gr < R) {
                        const RowInfo ri = rows[gr];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int j = j0 + 8 * c + e;
                            re[e] = 0.f; im[e] = 0.f;
                            if (j < p1) {
                                const uint4 pj = pu[j];
                                float cs, sn;
                                phase((uint32_t)ri.my * pj.y + (uint32_t)ri.mz * pj.z, cs, sn);
                                const float qj = __uint_as_float(pj.w);
                                re[e] = qj * cs; im[e] = qj * sn;
                            }
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) { re[e] = 0.f; im[e] = 0.f; }
                    }
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split2<BF>(re[2 * e], re[2 * e + 1], h[e], l[e]);
                    st16(ahi, tile_off(rl, c, kchunks), h[0], h[1], h[2], h[3]);
                    st16(alo, tile_off(rl, c, kchunks), l[0], l[1], l[2], l[3]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) split2<BF>(im[2 * e], im[2 * e + 1], h[e], l[e]);
                    st16(ahi, tile_off(64 + rl, c, kchunks), h[0], h[1], h[2], h[3]);
                    st16(alo, tile_off(64 + rl, c, kchunks), l[0], l[1], l[2], l[3]);
                }
            }
            // B: X_j[m] = e^{i k_x x_j}: column m = Re, column k_max + m = Im (m >= 1)
            unsigned char *bhi = st + kFMT * 2 * A_BYTES;
            unsigned char *blo = bhi + B_BYTES;
#pragma unroll 1
            for (int unit = t; unit < (kmax + 1) * kchunks; unit += 128) {
                const int m = unit / kchunks, c = unit % kchunks;
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = j0 + 8 * c + e;
                    re[e] = 0.f; im[e] = 0.f;
                    if (j < p1) {
                        const uint4 pj = pu[j];
                        phase((uint32_t)m * pj.x, re[e], im[e]);
                    }
                }
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split2<BF>(re[2 * e], re[2 * e + 1], h[e], l[e]);
                st16(bhi, tile_off(m, c, kchunks), h[0], h[1], h[2], h[3]);
                st16(blo, tile_off(m, c, kchunks), l[0], l[1], l[2], l[3]);
                if (m >= 1) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) split2<BF>(im[2 * e], im[2 * e + 1], h[e], l[e]);
                    st16(bhi, tile_off(kmax + m, c, kchunks), h[0], h[1], h[2], h[3]);
                    st16(blo, tile_off(kmax + m, c, kchunks), l[0], l[1], l[2], l[3]);
                }
            }
            fence_async_smem();
            mb_arrive(&full[s]);
        }
    } else if (warp == 4) {
        // ---- MMA issuer: the whole warp follows the loop, lane 0 issues ----
        const uint32_t idesc = idesc_f16(128, NF, BF);
        const uint32_t sbo = kchunks * 128;
        for (int it = 0; it < nst; ++it) {
            const int s = it % kFStages, u = it / kFStages;
            if (!waitw(&full[s], u & 1, abort)) break;
            tc_after();
            if (lane == 0) {
                const uint32_t st = su32(sm + s * STAGE);
                const uint32_t bhi = st + kFMT * 2 * A_BYTES, blo = bhi + B_BYTES;
#pragma unroll 1
                for (int mt = 0; mt < kFMT; ++mt) {
                    const uint32_t ahi = st + (mt * 2) * A_BYTES, alo = ahi + A_BYTES;
                    const uint32_t d = tmem + mt * 128;
#pragma unroll
                    for (int kk = 0; kk < kFK / 16; ++kk) {
                        const uint32_t o = kk * 256;
                        umma(d, sdesc(ahi + o, 128, sbo), sdesc(bhi + o, 128, sbo), idesc, (it | kk) != 0);
                        umma(d, sdesc(ahi + o, 128, sbo), sdesc(blo + o, 128, sbo), idesc, 1);
                        umma(d, sdesc(alo + o, 128, sbo), sdesc(bhi + o, 128, sbo), idesc, 1);
                    }
                }
                umma_commit(&empty[s]);
            }
            __syncwarp();
        }
        if (lane == 0) umma_commit(accf);
        __syncwarp();
    }

    // ---- epilogue: TMEM -> partials ----
    if (t < 128) {
        const bool ok = waitw(accf, 0, abort);
        tc_after();
        const int row = t;
#pragma unroll 1
        for (int mt = 0; mt < kFMT; ++mt) {
            const int gr = (mgroup * kFMT + mt) * 64 + (row & 63);
            const bool im_row = row >= 64;
#pragma unroll 1
            for (int c0 = 0; c0 < NF; c0 += 16) {
                float v[16];
                tm_ld16(tmem + ((uint32_t)(warp * 32) << 16) + mt * 128 + c0, v);
                if (!ok || gr >= R) continue;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int col = c0 + jj;
                    int m, comp;
                    if (col <= kmax) { m = col; comp = im_row ? 2 : 0; }
                    else if (col <= 2 * kmax) { m = col - kmax; comp = im_row ? 3 : 1; }
                    else continue;
                    spart[(((int64_t)ks * R + gr) * (kmax + 1) + m) * 4 + comp] = v[jj];
                }
            }
            if (ok && gr < R) spart[(((int64_t)ks * R + gr) * (kmax + 1)) * 4 + (im_row ? 3 : 1)] = 0.f;
        }
    }
    if (t == 0 && *abort) atomicOr(status, kStTimeout);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tm_dealloc(tmem, 256);
}

// ---- coefficient max, packing of G' into FP16/BF16 split tiles --------------------------

__global__ void k_gmax(int64_t count, const float *__restrict__ g, int *__restrict__ gmax)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(g[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(gmax, __float_as_int(m));   // m >= 0: int order = float order
}

// btile layout [pass][kb][part: hi, lo][NP columns x kBK] in [col/8][k/8][8][8] core matrices.
template <bool BF>
__global__ void k_bpack(int R2, int ncol, int NP, int nkb, const float *__restrict__ g,
                        const int *__restrict__ gmax, float *__restrict__ gscale,
                        uint16_t *__restrict__ btile)
{
    const int kb = blockIdx.x, pass = blockIdx.y;
    float scale = 1.f;
    if (!BF) {
        const float mx = __int_as_float(*gmax);
        if (mx > 0.f) scale = exp2f((float)(14 - ilogbf(mx)));
    }
    if (kb == 0 && pass == 0 && threadIdx.x == 0) gscale[0] = 1.f / scale;
    uint16_t *out = btile + ((int64_t)pass * nkb + kb) * 2 * NP * kBK;
    for (int e = threadIdx.x; e < NP * kBK; e += blockDim.x) {
        const int col = e / kBK, k = e % kBK;
        const int gk = kb * kBK + k, gc = pass * NP + col;
        float v = 0.f;
        if (gk < R2 && gc < ncol) v = g[(int64_t)gk * ncol + gc] * scale;
        uint32_t h, l;
        split2<BF>(v, 0.f, h, l);
        const int off = ((col >> 3) * (kBK / 8) + (k >> 3)) * 64 + (col & 7) * 8 + (k & 7);
        out[off] = (uint16_t)(h & 0xffffu);
        out[NP * kBK + off] = (uint16_t)(l & 0xffffu);
    }
}

// ---- back-scatter -----------------------------------------------------------------------
// grid (particle tiles of kBMT * 128, passes); block kBThreads.
// bpart layout [pass][n][4] = partial (F_x, F_y, F_z, phi) before q_i, 2 pi / L and scale.
template <bool BF>
__global__ void __launch_bounds__(kBThreads, 1)
k_bs_tc(int n, int R, int kmax, int ncol, int NP, int nkb, const RowInfo *__restrict__ rows,
        const uint4 *__restrict__ pu, const uint16_t *__restrict__ btile,
        float *__restrict__ bpart, int *__restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int A_BYTES = 128 * kBK * 2;          // 8 KB
    const int B_BYTES = NP * kBK * 2;
    const int STAGE = kBMT * 2 * A_BYTES + 2 * B_BYTES;
    uint64_t *full_a = reinterpret_cast<uint64_t *>(sm + kBStages * STAGE);
    uint64_t *full_b = full_a + kBStages;
    uint64_t *empty = full_b + kBStages;
    uint64_t *accf = empty + kBStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    int *coldesc = const_cast<int *>(reinterpret_cast<volatile int *>(tslot + 2));

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int pass = blockIdx.y;
    const int base = blockIdx.x * (kBMT * 128);
    const int kchunks = kBK / 8;
    const int NB = 2 * kmax + 1;

    if (t == 0) {
        for (int s = 0; s < kBStages; ++s) {
            mb_init(&full_a[s], 128); mb_init(&full_b[s], 1); mb_init(&empty[s], 1);
        }
        mb_init(accf, 1);
        *abort = 0;
        mb_fence_init();
    }
    // column descriptors of this pass: bits 0-7 m, 8-9 kind (0: m = 0, 1: first, 2: second),
    // 10-11 block (x, y, z), bit 12 padding
    for (int col = t; col < NP; col += kBThreads) {
        const int gc = pass * NP + col;
        int d = 1 << 12;
        if (gc < ncol) {
            const int blk = gc / NB, c = gc % NB;
            const int m = (c + 1) / 2;
            const int kind = c == 0 ? 0 : ((c & 1) ? 1 : 2);
            d = m | (kind << 8) | (blk << 10);
        }
        coldesc[col] = d;
    }
    if (warp == 0) { tm_alloc(tslot, 512); tm_relinquish(); }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    if (t < 128) {
        // ---- producers: P_i[r] = e^{i (k_y y_i + k_z z_i)} for two particles per thread ----
        uint32_t uy[kBMT], uz[kBMT];
        bool valid[kBMT];
#pragma unroll
        for (int mt = 0; mt < kBMT; ++mt) {
            const int i = base + mt * 128 + t;
            valid[mt] = i < n;
            const uint4 pi = pu[valid[mt] ? i : 0];
            uy[mt] = pi.y; uz[mt] = pi.z;
        }
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kBStages, u = kb / kBStages;
            if (u > 0 && !waitw(&empty[s], (u - 1) & 1, abort)) break;
            unsigned char *st = sm + s * STAGE;
            const int r0 = kb * (kBK / 2);
#pragma unroll 1
            for (int c = 0; c < kchunks; ++c) {
                int my[4], mz[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = r0 + 4 * c + e;
                    if (r < R) { const RowInfo ri = rows[r]; my[e] = ri.my; mz[e] = ri.mz; }
                    else { my[e] = 0; mz[e] = 0; }
                }
#pragma unroll
                for (int mt = 0; mt < kBMT; ++mt) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = r0 + 4 * c + e;
                        float cs = 0.f, sn = 0.f;
                        if (r < R && valid[mt])
                            phase((uint32_t)my[e] * uy[mt] + (uint32_t)mz[e] * uz[mt], cs, sn);
                        v[2 * e] = cs; v[2 * e + 1] = sn;
                    }
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) split2<BF>(v[2 * e], v[2 * e + 1], h[e], l[e]);
                    unsigned char *ahi = st + (mt * 2) * A_BYTES;
                    st16(ahi, tile_off(t, c, kchunks), h[0], h[1], h[2], h[3]);
                    st16(ahi + A_BYTES, tile_off(t, c, kchunks), l[0], l[1], l[2], l[3]);
                }
            }
            fence_async_smem();
            mb_arrive(&full_a[s]);
        }
    } else if (warp == 4) {
        // ---- TMA producer for the G' tiles: the whole warp follows the loop, lane 0 issues ----
        const uint32_t bytes = 2u * (uint32_t)B_BYTES;
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kBStages, u = kb / kBStages;
            if (u > 0 && !waitw(&empty[s], (u - 1) & 1, abort)) break;
            if (lane == 0) {
                unsigned char *dst = sm + s * STAGE + kBMT * 2 * A_BYTES;
                mb_expect_tx(&full_b[s], bytes);
                tma_bulk(dst, btile + ((int64_t)pass * nkb + kb) * 2 * NP * kBK, bytes, &full_b[s]);
            }
            __syncwarp();
            issued = kb + 1;
        }
        // every copy issued must have landed before the CTA can leave (bounded)
        for (int kb = issued - kBStages < 0 ? 0 : issued - kBStages; kb < issued; ++kb) {
            volatile int no_abort = 0;
            waitw(&full_b[kb % kBStages], (kb / kBStages) & 1, &no_abort);
        }
    } else if (warp == 5) {
        // ---- MMA issuer: the whole warp follows the loop, lane 0 issues ----
        const uint32_t idesc = idesc_f16(128, NP, BF);
        const uint32_t sbo = kchunks * 128;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kBStages, u = kb / kBStages;
            if (!waitw(&full_a[s], u & 1, abort)) break;
            if (!waitw(&full_b[s], u & 1, abort)) break;
            tc_after();
            if (lane == 0) {
                const uint32_t st = su32(sm + s * STAGE);
                const uint32_t bhi = st + kBMT * 2 * A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
                for (int mt = 0; mt < kBMT; ++mt) {
                    const uint32_t ahi = st + (mt * 2) * A_BYTES, alo = ahi + A_BYTES;
                    const uint32_t d = tmem + mt * 256;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t o = kk * 256;
                        umma(d, sdesc(ahi + o, 128, sbo), sdesc(bhi + o, 128, sbo), idesc, (kb | kk) != 0);
                        umma(d, sdesc(ahi + o, 128, sbo), sdesc(blo + o, 128, sbo), idesc, 1);
                        umma(d, sdesc(alo + o, 128, sbo), sdesc(bhi + o, 128, sbo), idesc, 1);
                    }
                }
                umma_commit(&empty[s]);
            }
            __syncwarp();
        }
        if (lane == 0) umma_commit(accf);
        __syncwarp();
    }

    // ---- epilogue: per particle, combine the accumulator row with X_i[m] ----
    if (t < 128) {
        const bool ok = waitw(accf, 0, abort);
        tc_after();
        // X table in the (now idle) stage buffers: xt[m * 128 + t]
        float2 *xt = reinterpret_cast<float2 *>(sm);
#pragma unroll 1
        for (int mt = 0; mt < kBMT; ++mt) {
            const int i = base + mt * 128 + t;
            const uint32_t ux = pu[i < n ? i : 0].x;
            for (int m = 0; m <= kmax; ++m) {
                float cs, sn;
                phase((uint32_t)m * ux, cs, sn);
                xt[m * 128 + t] = make_float2(cs, sn);
            }
            float fx = 0.f, fy = 0.f, fz = 0.f, ph = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < NP; c0 += 16) {
                float v[16];
                tm_ld16(tmem + ((uint32_t)(warp * 32) << 16) + mt * 256 + c0, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int d = coldesc[c0 + jj];
                    if (d & (1 << 12)) continue;
                    const int m = d & 0xff, kind = (d >> 8) & 3, blk = (d >> 10) & 3;
                    const float2 x = xt[m * 128 + t];
                    const float val = v[jj];
                    if (blk == 0) {
                        if (kind == 0) ph += val;
                        else if (kind == 1) { fx += (float)m * x.x * val; ph -= x.y * val; }
                        else { fx += (float)m * x.y * val; ph += x.x * val; }
                    } else {
                        const float w = kind == 0 ? val : (kind == 1 ? x.x * val : x.y * val);
                        if (blk == 1) fy += w; else fz += w;
                    }
                }
            }
            if (ok && i < n) {
                float4 *o = reinterpret_cast<float4 *>(bpart) + ((int64_t)pass * n + i);
                *o = make_float4(fx, fy, fz, ph);
            }
        }
    }
    if (t == 0 && *abort) atomicOr(status, kStTimeout);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tm_dealloc(tmem, 512);
}

// Sum the passes (fixed order) into the sorted reciprocal forces.
__global__ void k_bs_reduce(int64_t n, int npass, const float *__restrict__ bpart,
                            const double4_32a *__restrict__ pg, const float *__restrict__ gscale,
                            double L, double *__restrict__ f)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double qf = pg[s].w * (2.0 * kPi / L) * (double)gscale[0];
    double a[3] = {0.0, 0.0, 0.0};
    for (int ps = 0; ps < npass; ++ps) {
        const float4 v = reinterpret_cast<const float4 *>(bpart)[(int64_t)ps * n + s];
        a[0] += v.x; a[1] += v.y; a[2] += v.z;
    }
    f[3 * s + 0] = qf * a[0];
    f[3 * s + 1] = qf * a[1];
    f[3 * s + 2] = qf * a[2];
}

// ---- plan-side state ----------------------------------------------------------------------

struct TcState {
    int nf = 0;           // forward N (2 k_max + 1 rounded up to 16)
    int mgroups = 0;      // forward M groups
    int ks = 0;           // forward K splits
    int per = 0;          // forward particles per split
    int ncol = 0;         // back-scatter columns 3 (2 k_max + 1)
    int npass = 0, np = 0, nkb = 0;
    float *spart = nullptr;     // [ks][R][k+1][4]
    float *gmat = nullptr;      // [2R][ncol]
    int *gmax = nullptr;
    float *gscale = nullptr;
    uint16_t *btile = nullptr;  // [npass][nkb][2][np * kBK]
    float *bpart = nullptr;     // [npass][n][4]
};

void tc_shape(const Plan &p, int64_t n, TcState &s)
{
    s.nf = 16 * ((2 * p.kmax + 1 + 15) / 16);
    const int tiles = (p.R + 63) / 64;
    s.mgroups = (tiles + kFMT - 1) / kFMT;
    const int nblk = (int)((n + kFK - 1) / kFK);
    int want = (2 * 152 + s.mgroups - 1) / s.mgroups;
    if (want > nblk) want = nblk;
    if (want < 1) want = 1;
    const int blk_per = (nblk + want - 1) / want;
    s.per = blk_per * kFK;
    s.ks = (nblk + blk_per - 1) / blk_per;
    s.ncol = 3 * (2 * p.kmax + 1);
    s.npass = (s.ncol + kPassMax - 1) / kPassMax;
    s.np = 16 * (((s.ncol + s.npass - 1) / s.npass + 15) / 16);
    s.nkb = (2 * p.R + kBK - 1) / kBK;
}

size_t fwd_smem(int nf) { return (size_t)kFStages * (kFMT * 2 * 128 * kFK * 2 + 2 * nf * kFK * 2) + 256; }
size_t bs_smem(int np)
{
    size_t stage = (size_t)kBMT * 2 * 128 * kBK * 2 + 2 * (size_t)np * kBK * 2;
    return kBStages * stage + 256 + 4 * (size_t)np;
}

template <bool BF>
cudaError_t launch_bf(Plan &p, int64_t n, cudaStream_t st)
{
    TcState &s = *static_cast<TcState *>(p.tc);
    Workspace &ws = p.ws;
    cudaError_t e;
    prof_mark(p, kEvRecipStart, st);
    const size_t fs = fwd_smem(s.nf);
    if ((e = cudaFuncSetAttribute(k_fwd_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs)) != cudaSuccess)
        return e;
    k_fwd_tc<BF><<<dim3(s.mgroups, s.ks), kFThreads, fs, st>>>((int)n, p.R, p.kmax, s.nf, s.per,
                                                               p.rows_d, ws.pu, s.spart, p.d_status);
    prof_mark(p, kEvFwdEnd, st);
    if ((e = launch_sreduce_f32(p, s.ks, s.spart, s.gmat, s.ncol, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.gmax, 0, sizeof(int), st)) != cudaSuccess) return e;
    k_gmax<<<152, 256, 0, st>>>((int64_t)2 * p.R * s.ncol, s.gmat, s.gmax);
    k_bpack<BF><<<dim3(s.nkb, s.npass), 256, 0, st>>>(2 * p.R, s.ncol, s.np, s.nkb, s.gmat, s.gmax,
                                                      s.gscale, s.btile);
    prof_mark(p, kEvCoefEnd, st);
    const size_t bs = bs_smem(s.np);
    if ((e = cudaFuncSetAttribute(k_bs_tc<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs)) != cudaSuccess)
        return e;
    const int ptiles = (int)((n + kBMT * 128 - 1) / (kBMT * 128));
    k_bs_tc<BF><<<dim3(ptiles, s.npass), kBThreads, bs, st>>>((int)n, p.R, p.kmax, s.ncol, s.np, s.nkb,
                                                              p.rows_d, ws.pu, s.btile, s.bpart,
                                                              p.d_status);
    k_bs_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s.npass, s.bpart, ws.pg, s.gscale,
                                                            p.L, ws.f_recip);
    prof_mark(p, kEvBackEnd, st);
    p.launches += 6;
    return cudaGetLastError();
}

}  // namespace

size_t recip_tc_bytes(const Plan &p, int64_t n)
{
    TcState s;
    tc_shape(p, n, s);
    size_t b = 0;
    b += (size_t)s.ks * p.R * (p.kmax + 1) * 4 * sizeof(float);
    b += (size_t)2 * p.R * s.ncol * sizeof(float);
    b += (size_t)s.npass * s.nkb * 2 * s.np * kBK * sizeof(uint16_t);
    b += (size_t)s.npass * n * 4 * sizeof(float);
    return b + 64;
}

cudaError_t alloc_recip_tc(Plan &p, int64_t n)
{
    free_recip_tc(p);
    TcState *s = new TcState();
    tc_shape(p, n, *s);
    p.tc = s;
    cudaStream_t st = p.side_stream;
    cudaError_t e;
    if ((e = pool_alloc((void **)&s->spart, (size_t)s->ks * p.R * (p.kmax + 1) * 4 * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gmat, (size_t)2 * p.R * s->ncol * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gmax, 64, st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gscale, 64, st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->btile, (size_t)s->npass * s->nkb * 2 * s->np * kBK * sizeof(uint16_t), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->bpart, (size_t)s->npass * n * 4 * sizeof(float), st)) != cudaSuccess) return e;
    return cudaSuccess;
}

void free_recip_tc(Plan &p)
{
    TcState *s = static_cast<TcState *>(p.tc);
    if (!s) return;
    cudaStream_t st = p.side_stream;
    pool_free(s->spart, st); pool_free(s->gmat, st); pool_free(s->gmax, st);
    pool_free(s->gscale, st); pool_free(s->btile, st); pool_free(s->bpart, st);
    delete s;
    p.tc = nullptr;
}

cudaError_t launch_recip_tc(Plan &p, int64_t n, cudaStream_t st)
{
    if (!p.tc) return cudaErrorInvalidValue;
    if (p.precision == EWALD_MIXED_BF16) return launch_bf<true>(p, n, st);
    return launch_bf<false>(p, n, st);
}

}  // namespace ew
