// Reciprocal-space sum on the tcgen05 tensor cores (hot-path steps a5-a8, EWALD_MIXED and
// EWALD_MIXED_BF16).
//
// The two matrix-vector products of Eq. 3 (Algorithm 1: rho_hat_k from all particles;
// Algorithm 2: forces from all k) are evaluated as real matrix products on the tensor cores,
// with the k vectors grouped in rows r = (m_y, m_z) and m_x along the row (the row/column
// algebra, including the pairing of +m_x with -m_x, is documented in recip_simt.cu):
//
//   forward  (a6):  D_f[(Re|Im) A[r], col] = sum_j A_j[r] X_j[col]
//                   A_j[r] = e^{i(k_y y_j + k_z z_j)},  X_j carries q_j;  cols: Re X_j[0],
//                   then Re X_j[m], Im X_j[m] for m = 1..k_max (column 2m - 1 and 2m), so
//                   the first 2 m + 1 columns hold |m_x| <= m;  M = 2R, N = 2 k_max + 1,
//                   K = particles.  Rows run in order of decreasing n_x,max, and every
//                   tile of 64 rows multiplies only the columns its first row needs.
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
// Accumulation accuracy.  The rounding error of the tensor cores' FP32 accumulation grows
// with the number of products summed into one accumulator, so the forward product (a sum
// over all particles) accumulates only 128 particles per TMEM accumulator: two accumulator
// buffers alternate (one where tensor memory is short), and drain warps add every finished
// buffer into an FP32 running sum, rounded to nearest, that is kept in another region of
// tensor memory while the tensor cores fill the other buffer.  The back-scatter
// (a sum over rows) processes rows in order of decreasing m_y^2 + m_z^2, so the coefficients
// grow along the sum.
//
// Kernel structure (warp-specialised, mbarrier pipeline in shared memory):
//   forward:      warps 0-7 generate A of each stage; warps 8-11 drain TMEM; warps 12 and
//                 13 stream the particle data and the pre-built B operand of each stage by
//                 bulk TMA into two separate rings; warp 14 issues tcgen05.mma (one thread)
//                 and releases stages with tcgen05.commit.  Work is split evenly over one
//                 CTA per SM ("stream-K" over (row group, particle stage) items).
//   back-scatter: warps 0-7 generate A (one particle per thread) and then run the
//                 epilogue; warp 8 streams the pre-packed G' tiles (with their row headers)
//                 by bulk TMA; warp 9 issues tcgen05.mma.
// Shared-memory operand layout (no swizzle, K-major): 8x8 core matrices of 128 contiguous
// bytes, ordered [row / 8][k / 8][row % 8][k % 8]; descriptor LBO = 128 B (next core matrix
// along K), SBO = (K_stage / 8) * 128 B (next 8-row group).
// Every mbarrier wait is bounded (~1 s of globaltimer); a timeout sets a status bit and lets
// every role leave its loop; copies in flight and the last MMAs are waited for before the
// CTA releases TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ewald_internal.cuh"

namespace ew {
namespace {

// ---- tiling ---------------------------------------------------------------------------
constexpr int kFK = 32;        // forward: particles (K) per stage
constexpr int kFChunk = 4;     // forward: stages per TMEM accumulator (128 particles)
constexpr int kFThreads = 608; // forward: 19 warps
constexpr int kBK = 32;        // back-scatter: real K per stage (16 rows r)
constexpr int kBStages = 3;
constexpr int kBMT = 2;        // back-scatter: M tiles of 128 particles per CTA
constexpr int kBThreads = 320; // back-scatter: 10 warps
constexpr int kPassMax = 256;  // N columns per back-scatter pass (one MMA)
constexpr int kHdr = 128;      // row header of every packed G' K-block: 16 x (m_y, m_z)

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
// try_wait with a suspend-time hint: a waiting thread sleeps in hardware (up to ~20 us)
// until the phase completes instead of re-issuing the poll
__device__ __forceinline__ uint32_t mb_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su32(b)), "r"(parity), "r"(20000u) : "memory");
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
// Transposed product.  A tcgen05.mma of M = 128, K = 16 takes the same time whatever its N
// (up to 256), so the wide dimension of the forward product goes to N: per 32-particle stage,
//   D[c, n] += sum_j X_j[c] P_j[n],   c = column (m_x slot, the MMA's M, from the pre-built
//   operand), n = 0..127: Re P_j of row n, n = 128..255: Im P_j of row n - 128 (the MMA's N,
//   generated by the producers), P_j[r] = e^{i(k_y y_j + k_z z_j)}.
// Rows run in forward order (decreasing n_x,max) in groups of 128.  A group needs the columns
// |m_x| <= n_x,max of its first row; where that is more than 128 columns, it is processed as
// two "virtual groups" (column passes 0 and 1), each with one M tile of 128 columns.
//
// Work partition ("stream-K"): the items are (virtual group v, stage s), W = nvg * stages of
// them in v-major order, and CTA c of the G CTAs (one per SM) takes the items
// [floor(c W / G), floor((c + 1) W / G)).  A CTA's items form segments, each inside one
// virtual group; every segment yields one partial sum ("piece"), written to
// dpart[((v * maxp + piece) * 128 + c) * 256 + n] with piece = c - (first CTA of the group).
//
// Roles (block kFThreads = 19 warps):
//   warps 0-7    producers: P of every stage (128 rows x 32 particles, Re and Im, hi and lo
//                terms) into the P ring; particle coordinates come from the coordinate ring
//   warps 8-15   drain: every kFChunk stages (128 particles) the TMEM accumulator
//                (columns 0-255) is added into an FP32 running sum in TMEM columns 256-511;
//                at the end of a segment the sum goes to dpart.  Warp 8 + q and 12 + q own
//                TMEM lanes 32q..32q+31, columns 0-127 and 128-255 respectively.
//   warp 16      bulk copies of (u_y, u_z) of every stage into the coordinate ring
//   warp 17      bulk copies of the column operand (q_j X_j[c], hi and lo) into the X ring
//   warp 18      tcgen05.mma issue (one thread) and stage release by tcgen05.commit
__host__ __device__ inline int64_t fwd_item0(int c, int64_t W, int G) { return (int64_t)c * W / G; }
__host__ __device__ inline int fwd_cta_of(int64_t w, int64_t W, int G) { return (int)(((w + 1) * G - 1) / W); }

// Position in a ring of `depth` slots: slot index and the number of completed laps.
struct RingPos {
    int slot = 0, lap = 0;
    __device__ __forceinline__ void next(int depth) { if (++slot == depth) { slot = 0; ++lap; } }
};

__device__ __forceinline__ void tm_ld16r(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                   "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_st16r(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]),
                   "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]),
                   "r"(r[13]), "r"(r[14]), "r"(r[15]) : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Split a pair of FP32 values into packed FP16 hi and lo pairs: hi = rn(v), lo = rn(v - hi)
// (v - hi is exact in FP32; the mixed-precision FMA forms it from the packed hi directly).
__device__ __forceinline__ void split2_f16(float a, float b, uint32_t &hi, uint32_t &lo)
{
    __half2 h = __floats2half2_rn(a, b);
    const unsigned short h0 = __half_as_ushort(__low2half(h)), h1 = __half_as_ushort(__high2half(h));
    const unsigned short m1 = 0xbc00;          // -1.0 in FP16
    float la, lb;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(la) : "h"(h0), "h"(m1), "f"(a));
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(lb) : "h"(h1), "h"(m1), "f"(b));
    __half2 l = __floats2half2_rn(la, lb);
    hi = *reinterpret_cast<uint32_t *>(&h);
    lo = *reinterpret_cast<uint32_t *>(&l);
}

template <bool BF>
__device__ __forceinline__ void split2x(float a, float b, uint32_t &hi, uint32_t &lo)
{
    if (BF) split2<true>(a, b, hi, lo);
    else split2_f16(a, b, hi, lo);
}

// Virtual group descriptor: x = first forward row, y = column pass, z = columns (multiple of
// 16, <= 128) copied for this pass.
template <bool BF>
__global__ void __launch_bounds__(kFThreads, 1)
k_fwd_tc(int R, int NF, int nst_all, int64_t W, int maxp, int SA, int SX, int SP, int KCH,
         const int4 *__restrict__ vgs, const RowInfo *__restrict__ rows,
         const int *__restrict__ fperm, const uint2 *__restrict__ yz,
         const unsigned char *__restrict__ bblob, float *__restrict__ dpart,
         int *__restrict__ status)
{
    constexpr int KC = kFK / 8;                  // K chunks of 8 per stage
    constexpr int P_HALF = 256 * kFK * 2;        // one term of the phase tile: 256 rows x 32
    constexpr int P_STAGE = 2 * P_HALF;          // hi and lo
    constexpr int X_HALF = 128 * kFK * 2;        // one term of the column tile: 128 x 32
    constexpr int X_STAGE = 2 * X_HALF;
    constexpr int C_STAGE = kFK * 8;             // (u_y, u_z) of 32 particles
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *smP = sm;
    unsigned char *smX = smP + SA * P_STAGE;
    unsigned char *smC = smX + SX * X_STAGE;
    uint64_t *a_full = reinterpret_cast<uint64_t *>(smC + SP * C_STAGE);
    uint64_t *a_empty = a_full + SA;
    uint64_t *x_full = a_empty + SA;
    uint64_t *x_empty = x_full + SX;
    uint64_t *c_full = x_empty + SX;
    uint64_t *c_empty = c_full + SP;
    uint64_t *accf = c_empty + SP;
    uint64_t *acce = accf + 1;
    uint64_t *mmad = acce + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mmad + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int G = gridDim.x, c = blockIdx.x;
    const int64_t w_begin = fwd_item0(c, W, G), w_end = fwd_item0(c + 1, W, G);
    const int nit = (int)(w_end - w_begin);
    const int v0 = (int)(w_begin / nst_all), s0 = (int)(w_begin % nst_all);

    if (t == 0) {
        // producer barriers count one arrival per producer warp (lane 0, after the warp's
        // stores are fenced for the async proxy and the warp has synchronised)
        for (int s = 0; s < SA; ++s) { mb_init(&a_full[s], 8); mb_init(&a_empty[s], 1); }
        for (int s = 0; s < SX; ++s) { mb_init(&x_full[s], 1); mb_init(&x_empty[s], 1); }
        for (int s = 0; s < SP; ++s) { mb_init(&c_full[s], 1); mb_init(&c_empty[s], 8); }
        mb_init(accf, 1);
        mb_init(acce, 256);
        mb_init(mmad, 1);
        *abort = 0;
        mb_fence_init();
    }
    if (warp == 0) { tm_alloc(tslot, 512); tm_relinquish(); }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    if (t < 256) {
        // ---- producers: thread t owns row rl = t % 128 and particles 16h..16h+15 ----
        const int rl = t & 127, h = t >> 7;
        int my = 0, mz = 0;
        int vcur = -1;
        int v = v0, sg = s0;
        RingPos ra, rp;
        for (int it = 0; it < nit; ++it, ++sg, ra.next(SA), rp.next(SP)) {
            if (sg == nst_all) { sg = 0; ++v; }
            if (v != vcur) {
                vcur = v;
                const int fr = vgs[v].x + rl;
                my = 0; mz = 0;                    // padding rows: any finite phase
                if (fr < R) { const RowInfo ri = rows[fperm[fr]]; my = ri.my; mz = ri.mz; }
            }
            if (ra.lap > 0 && !waitw(&a_empty[ra.slot], (ra.lap - 1) & 1, abort)) break;
            if (!waitw(&c_full[rp.slot], rp.lap & 1, abort)) break;
            uint32_t py[16], pz[16];
            {
                const uint4 *C4 = reinterpret_cast<const uint4 *>(smC + rp.slot * C_STAGE) + 8 * h;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint4 q4 = C4[i];
                    py[2 * i] = q4.x; pz[2 * i] = q4.y; py[2 * i + 1] = q4.z; pz[2 * i + 1] = q4.w;
                }
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&c_empty[rp.slot]);
            float cs[16], sn[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) phase((uint32_t)my * py[e] + (uint32_t)mz * pz[e], cs[e], sn[e]);
            unsigned char *hi = smP + ra.slot * P_STAGE, *lo = hi + P_HALF;
#pragma unroll
            for (int q = 0; q < 2; ++q) {          // K chunk 2h + q: particles 16h + 8q ..
                uint32_t ch[4], cl[4], sh[4], sl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    split2x<BF>(cs[8 * q + 2 * e], cs[8 * q + 2 * e + 1], ch[e], cl[e]);
                    split2x<BF>(sn[8 * q + 2 * e], sn[8 * q + 2 * e + 1], sh[e], sl[e]);
                }
                const uint32_t ore = tile_off(rl, 2 * h + q, KC), oim = tile_off(128 + rl, 2 * h + q, KC);
                st16(hi, ore, ch[0], ch[1], ch[2], ch[3]);
                st16(lo, ore, cl[0], cl[1], cl[2], cl[3]);
                st16(hi, oim, sh[0], sh[1], sh[2], sh[3]);
                st16(lo, oim, sl[0], sl[1], sl[2], sl[3]);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mb_arrive(&a_full[ra.slot]);
        }
    } else if (t < 512) {
        // ---- drain: TMEM accumulator -> TMEM running sum -> dpart ----
        const int dq = warp & 3, dh = (warp - 8) >> 2;        // lane quadrant, column half
        const uint32_t lanes = (uint32_t)(dq * 32) << 16;
        const int cl = dq * 32 + lane;                         // this thread's column c
        int gch = 0;
        int64_t w = w_begin;
        bool ok = true;
        while (w < w_end && ok) {
            const int v = (int)(w / nst_all);
            const int64_t seg_end = min(w_end, (int64_t)(v + 1) * nst_all);
            const int nchs = (int)((seg_end - w + KCH - 1) / KCH);
            const int piece = c - fwd_cta_of((int64_t)v * nst_all, W, G);
            // warps whose 32 lanes (columns) are all past the pass's column count have
            // nothing to add (their sums are never read); they still take part in the
            // barrier handshake
            const bool work = dq * 32 < vgs[v].z;
            for (int k = 0; k < nchs; ++k, ++gch) {
                if (!waitw(accf, gch & 1, abort)) { ok = false; break; }
                tc_after();
#pragma unroll 1
                for (int c0 = 0; work && c0 < 128; c0 += 32) {
                    const uint32_t src = tmem + lanes + (uint32_t)(dh * 128 + c0);
                    const uint32_t dst = src + 256;
                    uint32_t a0[16], a1[16], s0v[16], s1v[16];
                    tm_ld16r(src, a0);
                    tm_ld16r(src + 16, a1);
                    if (k > 0) { tm_ld16r(dst, s0v); tm_ld16r(dst + 16, s1v); }
                    tm_wait_ld();
                    if (k > 0) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            a0[i] = __float_as_uint(__uint_as_float(s0v[i]) + __uint_as_float(a0[i]));
                            a1[i] = __float_as_uint(__uint_as_float(s1v[i]) + __uint_as_float(a1[i]));
                        }
                    }
                    tm_st16r(dst, a0);
                    tm_st16r(dst + 16, a1);
                }
                tm_wait_st();
                tc_before();
                mb_arrive(acce);
            }
            if (!ok) break;
            // the segment's partial sum -> dpart, columns c < the pass's column count only (the
            // TMEM loads are warp-wide; a warp whose lanes are all past the count skips them)
            const int ncv = vgs[v].z;
            if (dq * 32 < ncv) {
                float4 *o = reinterpret_cast<float4 *>(dpart + (((int64_t)v * maxp + piece) * 128 + cl) * 256 + dh * 128);
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += 16) {
                    uint32_t r[16];
                    tm_ld16r(tmem + lanes + (uint32_t)(256 + dh * 128 + c0), r);
                    tm_wait_ld();
                    if (cl < ncv) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            o[c0 / 4 + i] = make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                                        __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3]));
                    }
                }
            }
            w = seg_end;
        }
    } else if (warp == 16) {
        // ---- bulk copies: (u_y, u_z) of every stage ----
        int issued = 0;
        int sg = s0;
        RingPos rp;
        for (int it = 0; it < nit; ++it, ++sg, rp.next(SP)) {
            if (sg == nst_all) sg = 0;
            if (rp.lap > 0 && !waitw(&c_empty[rp.slot], (rp.lap - 1) & 1, abort)) break;
            if (lane == 0) {
                mb_expect_tx(&c_full[rp.slot], (uint32_t)C_STAGE);
                tma_bulk(smC + rp.slot * C_STAGE, yz + (int64_t)sg * kFK, (uint32_t)C_STAGE, &c_full[rp.slot]);
            }
            __syncwarp();
            issued = it + 1;
        }
        for (int it = issued - SP < 0 ? 0 : issued - SP; it < issued; ++it) {
            volatile int no_abort = 0;
            waitw(&c_full[it % SP], (it / SP) & 1, &no_abort);
        }
    } else if (warp == 17) {
        // ---- bulk copies: column operand (hi, lo) of every stage, this pass's columns ----
        const int B_BYTES = NF * kFK * 2;                      // one term of a stage of bblob
        int issued = 0;
        int v = v0, sg = s0;
        int4 vd = vgs[v];
        RingPos rx;
        for (int it = 0; it < nit; ++it, ++sg, rx.next(SX)) {
            if (sg == nst_all) { sg = 0; ++v; vd = vgs[v]; }
            if (rx.lap > 0 && !waitw(&x_empty[rx.slot], (rx.lap - 1) & 1, abort)) break;
            if (lane == 0) {
                const uint32_t part = (uint32_t)vd.z * kFK * 2;
                const unsigned char *src = bblob + (int64_t)sg * 2 * B_BYTES + (int64_t)vd.y * X_HALF;
                mb_expect_tx(&x_full[rx.slot], 2 * part);
                tma_bulk(smX + rx.slot * X_STAGE, src, part, &x_full[rx.slot]);
                tma_bulk(smX + rx.slot * X_STAGE + X_HALF, src + B_BYTES, part, &x_full[rx.slot]);
            }
            __syncwarp();
            issued = it + 1;
        }
        for (int it = issued - SX < 0 ? 0 : issued - SX; it < issued; ++it) {
            volatile int no_abort = 0;
            waitw(&x_full[it % SX], (it / SX) & 1, &no_abort);
        }
    } else if (warp == 18) {
        // ---- MMA issuer: D[c, n] += X[c, k] P[n, k], three split products per K step ----
        const uint32_t idesc = idesc_f16(128, 256, BF);
        const uint32_t sbo = KC * 128;
        int gch = -1;
        int sg = s0, ls = 0;                 // stage within the virtual group, index in segment
        RingPos ra, rx;
        for (int it = 0; it < nit; ++it, ++sg, ++ls, ra.next(SA), rx.next(SX)) {
            if (sg == nst_all) { sg = 0; ls = 0; }
            const bool first = (ls % KCH) == 0;
            const bool last = (ls % KCH) == KCH - 1 || sg == nst_all - 1 || it == nit - 1;
            if (first) ++gch;
            if (first && gch >= 1 && !waitw(acce, (gch - 1) & 1, abort)) break;
            if (!waitw(&a_full[ra.slot], ra.lap & 1, abort)) break;
            if (!waitw(&x_full[rx.slot], rx.lap & 1, abort)) break;
            tc_after();
            if (lane == 0) {
                const uint32_t phi = su32(smP + ra.slot * P_STAGE), plo = phi + P_HALF;
                const uint32_t xhi = su32(smX + rx.slot * X_STAGE), xlo = xhi + X_HALF;
#pragma unroll
                for (int kk = 0; kk < kFK / 16; ++kk) {
                    const uint32_t o = kk * 256;
                    umma(tmem, sdesc(xhi + o, 128, sbo), sdesc(phi + o, 128, sbo), idesc, (first && kk == 0) ? 0u : 1u);
                    umma(tmem, sdesc(xhi + o, 128, sbo), sdesc(plo + o, 128, sbo), idesc, 1);
                    umma(tmem, sdesc(xlo + o, 128, sbo), sdesc(phi + o, 128, sbo), idesc, 1);
                }
                umma_commit(&a_empty[ra.slot]);
                umma_commit(&x_empty[rx.slot]);
                if (last) umma_commit(accf);
            }
            __syncwarp();
        }
        if (lane == 0) umma_commit(mmad);
        __syncwarp();
        volatile int no_abort = 0;
        waitw(mmad, 0, &no_abort);
    }
    if (t == 0 && *abort) atomicOr(status, kStTimeout);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tm_dealloc(tmem, 512);
}

// ---- a5: B operand of the forward product, once per evaluation --------------------------
// For every 32-particle stage: yz[stage * 32 + j] = (u_y, u_z) of the particle (zero past n),
// and bblob[stage] = [hi: NF x 32][lo: NF x 32] with column 0 = Re(q_j X_j[0]), column
// 2m - 1 = Re(q_j X_j[m]), column 2m = Im(q_j X_j[m]) (m >= 1), zero padding columns, in the
// core-matrix layout;
// X_j[m] = e^{i 2 pi m x_j / L}.  Particles past n have zero charge, so their B rows vanish
// and the A rows the producers build for them (from (0, 0)) contribute nothing.
// grid: stages, block 256.
template <bool BF>
__global__ void k_xgen(int n, int kmax, int NF, const uint4 *__restrict__ pu,
                       uint2 *__restrict__ yz, unsigned char *__restrict__ bblob)
{
    constexpr int KC = kFK / 8;
    const int B_BYTES = NF * kFK * 2;
    const int stg = blockIdx.x;
    const int j0 = stg * kFK;
    unsigned char *bhi = bblob + (int64_t)stg * 2 * B_BYTES;
    if (threadIdx.x < kFK) {
        const int j = j0 + threadIdx.x;
        uint2 v = make_uint2(0u, 0u);
        if (j < n) { const uint4 p = pu[j]; v = make_uint2(p.y, p.z); }
        yz[j] = v;
    }
    for (int unit = threadIdx.x; unit < NF * KC; unit += blockDim.x) {
        const int col = unit / KC, cc = unit % KC;
        const bool im = col > 0 && (col & 1) == 0;     // column 2m: Im X[m]; 2m - 1: Re X[m]
        const int m = (col + 1) >> 1;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = j0 + 8 * cc + e;
            v[e] = 0.f;
            if (j < n && col <= 2 * kmax) {
                const uint4 pj = pu[j];
                float cs, sn;
                phase((uint32_t)m * pj.x, cs, sn);
                v[e] = __uint_as_float(pj.w) * (im ? sn : cs);
            }
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split2<BF>(v[2 * e], v[2 * e + 1], h[e], l[e]);
        st16(bhi, tile_off(col, cc, KC), h[0], h[1], h[2], h[3]);
        st16(bhi + B_BYTES, tile_off(col, cc, KC), l[0], l[1], l[2], l[3]);
    }
}

// ---- a6-a7: FP64 reduction of the forward partials, S(k), energy, G' ---------------------
// grid (tiles of 64 rows in forward order, m = 0..k_max); block 64 (one row per thread).
// The partial sums (pieces) of a tile are added in CTA order, so the result does not depend
// on timing.
// Writes S in K_half order, the energy of the 64 rows and one m as a fixed-order block sum
// e_part[m * ntiles + tile], the coefficient matrix column-major
// gmat_t[col * 2R + (2r | 2r + 1)], and the max |G'| (as int bits).
__global__ void __launch_bounds__(64)
k_sreduce_tc(int nst_all, int64_t W, int G, int maxp, const int2 *__restrict__ gvg, int ntiles,
             int R, int kmax, int NF, const RowInfo *__restrict__ rows,
             const int *__restrict__ fperm, const float *__restrict__ dpart,
             const double *__restrict__ gk, double *__restrict__ S, double *__restrict__ e_part,
             float *__restrict__ gmat_t, int *__restrict__ gmax)
{
    __shared__ double ered[2];
    const int tile = blockIdx.x, m = blockIdx.y, rl = threadIdx.x;
    const int fr = tile * 64 + rl;                  // row in forward order
    const int NB = 2 * kmax + 1;
    const int64_t R2 = 2 * (int64_t)R;
    float gm = 0.f;
    double e = 0.0;
    if (fr < R) {
        const int r = fperm[fr];                    // row index of the coefficient matrix
        const RowInfo ri = rows[r];
        const bool origin = ri.my == 0 && ri.mz == 0;
        const double wy = ri.my, wz = ri.mz;
        double t[4] = {0.0, 0.0, 0.0, 0.0};         // T_rr, T_ri, T_ir, T_ii
        const int cre = m == 0 ? 0 : 2 * m - 1, cim = 2 * m;   // columns of Re X[m], Im X[m]
        if (m <= ri.nxmax) {
            // the pieces of a column's virtual group: one per CTA that worked on it, in CTA
            // order; n = row in the group (Re P) and 128 + row (Im P)
            const int g = fr / 128, n = fr % 128;
            const int2 gv = gvg[g];
#pragma unroll
            for (int which = 0; which < 2; ++which) {
                if (which == 1 && m == 0) break;
                const int col = which == 0 ? cre : cim;
                const int v = gv.x + col / 128;
                const int npc = fwd_cta_of((int64_t)(v + 1) * nst_all - 1, W, G) -
                                fwd_cta_of((int64_t)v * nst_all, W, G) + 1;
                const float *o = dpart + ((int64_t)v * maxp * 128 + col % 128) * 256;
                double a = 0.0, b = 0.0;
#pragma unroll 4
                for (int pc = 0; pc < npc; ++pc, o += (int64_t)128 * 256) {
                    a += (double)o[n];
                    b += (double)o[128 + n];
                }
                if (which == 0) { t[0] = a; t[2] = b; } else { t[1] = a; t[3] = b; }
            }
        }
        const bool vp = m <= ri.nxmax && (!origin || m > 0);
        const bool vn = m >= 1 && m <= ri.nxmax && !origin;
        const double spr = t[0] - t[3], spi = t[2] + t[1];
        const double snr = t[0] + t[3], sni = t[2] - t[1];
        double gp = 0.0, gn = 0.0;
        if (vp) {
            const int idx = origin ? ri.koff + (m - 1) : ri.koff + ri.nxmax + m;
            gp = gk[idx];
            S[2 * (int64_t)idx] = spr; S[2 * (int64_t)idx + 1] = spi;
            e += gp * (spr * spr + spi * spi);
        }
        if (vn) {
            const int idx = ri.koff + ri.nxmax - m;
            gn = gk[idx];
            S[2 * (int64_t)idx] = snr; S[2 * (int64_t)idx + 1] = sni;
            e += gn * (snr * snr + sni * sni);
        }
        const double Gpr = vp ? 2.0 * gp * spr : 0.0, Gpi = vp ? -2.0 * gp * spi : 0.0;
        const double Gnr = vn ? 2.0 * gn * snr : 0.0, Gni = vn ? -2.0 * gn * sni : 0.0;
        float v[3][2][2];   // [block][column 1|2][re|im]
        int cols[2];
        if (m == 0) {
            cols[0] = 0; cols[1] = -1;
            v[0][0][0] = (float)Gpr;          v[0][0][1] = (float)(-Gpi);
            v[1][0][0] = (float)(wy * Gpi);   v[1][0][1] = (float)(wy * Gpr);
            v[2][0][0] = (float)(wz * Gpi);   v[2][0][1] = (float)(wz * Gpr);
        } else {
            cols[0] = 2 * m - 1; cols[1] = 2 * m;
            v[0][0][0] = (float)(Gpi - Gni);        v[0][0][1] = (float)(Gpr - Gnr);
            v[0][1][0] = (float)(Gpr + Gnr);        v[0][1][1] = (float)(-(Gpi + Gni));
            v[1][0][0] = (float)(wy * (Gpi + Gni)); v[1][0][1] = (float)(wy * (Gpr + Gnr));
            v[1][1][0] = (float)(wy * (Gpr - Gnr)); v[1][1][1] = (float)(-wy * (Gpi - Gni));
            v[2][0][0] = (float)(wz * (Gpi + Gni)); v[2][0][1] = (float)(wz * (Gpr + Gnr));
            v[2][1][0] = (float)(wz * (Gpr - Gnr)); v[2][1][1] = (float)(-wz * (Gpi - Gni));
        }
#pragma unroll
        for (int blk = 0; blk < 3; ++blk)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                if (cols[cc] < 0) continue;
                const int64_t col = blk * NB + cols[cc];
                *reinterpret_cast<float2 *>(gmat_t + col * R2 + 2 * r) = make_float2(v[blk][cc][0], v[blk][cc][1]);
                gm = fmaxf(gm, fmaxf(fabsf(v[blk][cc][0]), fabsf(v[blk][cc][1])));
            }
    }
    // fixed-order energy sum of the block (shuffle tree per warp, then warp 0 + warp 1)
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((rl & 31) == 0) ered[rl >> 5] = e;
    for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_down_sync(0xffffffffu, gm, o));
    if ((rl & 31) == 0) atomicMax(gmax, __float_as_int(gm));   // gm >= 0: int order = float order
    __syncthreads();
    if (rl == 0) e_part[(int64_t)m * ntiles + tile] = ered[0] + ered[1];
}

// Back-scatter column order: |m_x| = m major, so that a pass (a range of columns) needs only
// the rows with n_x,max >= the smallest m of its columns, a suffix of the row order.
// Column gc: gc < 3 -> m = 0, block gc; else u = gc - 3: m = 1 + u / 6, block (u % 6) / 2,
// kind 1 + (u & 1) (kind 1: coefficient column 2m - 1, kind 2: column 2m of the block).
struct BsCol { int m, kind, blk; };
// Passes: pass q holds columns [q kPassMax, min(ncol, (q + 1) kPassMax)), padded to 16, so all
// passes but the last use the full MMA width (an MMA costs the same whatever its N) and the
// last, narrow one has the largest m and the shortest row range.
__host__ __device__ inline int bs_pass_cols(int ncol, int pass)
{
    const int w = ncol - pass * kPassMax;
    return 16 * (((w < kPassMax ? w : kPassMax) + 15) / 16);
}
__host__ __device__ inline BsCol bs_col(int gc)
{
    if (gc < 3) return {0, 0, gc};
    const int u = gc - 3;
    return {1 + u / 6, 1 + (u & 1), (u % 6) / 2};
}

// Pack G' (column-major FP32) into split half-precision tiles with a row header:
// blob[pass][kb] = [16 x (m_y, m_z) int2][hi: NP x kBK][lo: NP x kBK], core-matrix layout.
// One thread packs 8 consecutive K of one column: one 16-byte store per part.
template <bool BF>
__global__ void k_bpack(int R, int ncol, int NPS, int nkb, const RowInfo *__restrict__ rows,
                        const float *__restrict__ gmat_t, const int *__restrict__ gmax,
                        float *__restrict__ gscale, unsigned char *__restrict__ blob)
{
    const int kb = blockIdx.x, pass = blockIdx.y;
    float scale = 1.f;
    if (!BF) {
        const float mx = __int_as_float(*gmax);
        if (mx > 0.f) scale = exp2f((float)(14 - ilogbf(mx)));
    }
    if (kb == 0 && pass == 0 && threadIdx.x == 0) gscale[0] = 1.f / scale;
    const int NP = bs_pass_cols(ncol, pass);            // columns of this pass
    const int64_t bsz = kHdr + 2 * (int64_t)NPS * kBK * 2;  // slot stride: the widest pass
    unsigned char *out = blob + ((int64_t)pass * nkb + kb) * bsz;
    if (threadIdx.x < kBK / 2) {
        const int r = kb * (kBK / 2) + threadIdx.x;
        int2 h = make_int2(0, 0);
        if (r < R) { const RowInfo ri = rows[r]; h = make_int2(ri.my, ri.mz); }
        reinterpret_cast<int2 *>(out)[threadIdx.x] = h;
    }
    unsigned char *hi = out + kHdr;
    unsigned char *lo = hi + NP * kBK * 2;
    const int64_t R2 = 2 * (int64_t)R;
    const int NB = ncol / 3;
    for (int u = threadIdx.x; u < NP * (kBK / 8); u += blockDim.x) {
        const int col = u / (kBK / 8), kc = u % (kBK / 8);
        const int gc = pass * kPassMax + col;
        const BsCol bc = bs_col(gc);
        const int64_t oc = (int64_t)bc.blk * NB + (bc.kind == 0 ? 0 : (bc.kind == 1 ? 2 * bc.m - 1 : 2 * bc.m));
        const int64_t gk0 = (int64_t)kb * kBK + 8 * kc;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            v[e] = (gk0 + e < R2 && gc < ncol) ? gmat_t[oc * R2 + gk0 + e] * scale : 0.f;
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split2<BF>(v[2 * e], v[2 * e + 1], h[e], l[e]);
        const uint32_t off = tile_off(col, kc, kBK / 8);
        st16(hi, off, h[0], h[1], h[2], h[3]);
        st16(lo, off, l[0], l[1], l[2], l[3]);
    }
}

// ---- back-scatter -----------------------------------------------------------------------
// grid (particle tiles of kBMT * 128, passes); block kBThreads.
// bpart layout [pass][n] float4 = partial (F_x, F_y, F_z, phi) before q_i, 2 pi / L and scale.
template <bool BF>
__global__ void __launch_bounds__(kBThreads, 1)
k_bs_tc(int n, int R, int kmax, int ncol, int NPS, int nkb, int4 kb0s, const uint4 *__restrict__ pu,
        const unsigned char *__restrict__ blob, float *__restrict__ bpart, int *__restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int KC = kBK / 8;
    const int A_BYTES = 128 * kBK * 2;          // 8 KB
    const int NP = bs_pass_cols(ncol, blockIdx.y);   // columns (MMA N) of this pass
    const int B_BYTES = NP * kBK * 2;
    const int BLOB = kHdr + 2 * B_BYTES;             // bytes copied per K block
    const int B_OFF = kBMT * 2 * A_BYTES;
    const int STAGE = B_OFF + kHdr + 2 * NPS * kBK * 2;   // stage layout sized for the widest pass
    const int64_t SLOT = kHdr + 2 * (int64_t)NPS * kBK * 2;
    uint64_t *full_a = reinterpret_cast<uint64_t *>(sm + kBStages * STAGE);
    uint64_t *full_b = full_a + kBStages;
    uint64_t *empty = full_b + kBStages;
    uint64_t *accf = empty + kBStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accf + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tslot + 1);
    int *coldesc = reinterpret_cast<int *>(tslot + 2);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int pass = blockIdx.y;
    const int base = blockIdx.x * (kBMT * 128);
    // first K block of this pass: rows before it have n_x,max below every m of the pass
    const int kb0 = pass == 0 ? kb0s.x : (pass == 1 ? kb0s.y : (pass == 2 ? kb0s.z : kb0s.w));

    if (t == 0) {
        for (int s = 0; s < kBStages; ++s) {
            mb_init(&full_a[s], 256); mb_init(&full_b[s], 1); mb_init(&empty[s], 1);
        }
        mb_init(accf, 1);
        *abort = 0;
        mb_fence_init();
    }
    // column descriptors of this pass: bits 0-7 m, 8-9 kind (0: m = 0, 1: first, 2: second),
    // 10-11 block (x, y, z), bit 12 padding
    for (int col = t; col < NP; col += kBThreads) {
        const int gc = pass * kPassMax + col;
        int d = 1 << 12;
        if (gc < ncol) {
            const BsCol bc = bs_col(gc);
            d = bc.m | (bc.kind << 8) | (bc.blk << 10);
        }
        coldesc[col] = d;
    }
    if (warp == 0) { tm_alloc(tslot, 512); tm_relinquish(); }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    if (t < 256) {
        // ---- producers: P_i[r] = e^{i (k_y y_i + k_z z_i)}, one particle per thread ----
        const int mt = t >> 7, row = t & 127;
        const int i = base + t;
        const bool valid = i < n;
        const uint4 pi = pu[valid ? i : 0];
        for (int kb = kb0; kb < nkb; ++kb) {
            const int s = (kb - kb0) % kBStages, u = (kb - kb0) / kBStages;
            if (u > 0 && !waitw(&empty[s], (u - 1) & 1, abort)) break;
            if (!waitw(&full_b[s], u & 1, abort)) break;      // row header of this K block
            unsigned char *st = sm + s * STAGE;
            const int2 *hdr = reinterpret_cast<const int2 *>(st + B_OFF);
            const int r0 = kb * (kBK / 2);
            unsigned char *ahi = st + (mt * 2) * A_BYTES;
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                float v[8];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int2 h = hdr[4 * c + e];
                    float cs = 0.f, sn = 0.f;
                    if (valid && r0 + 4 * c + e < R)
                        phase((uint32_t)h.x * pi.y + (uint32_t)h.y * pi.z, cs, sn);
                    v[2 * e] = cs; v[2 * e + 1] = sn;
                }
                uint32_t hh[4], ll[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split2<BF>(v[2 * e], v[2 * e + 1], hh[e], ll[e]);
                st16(ahi, tile_off(row, c, KC), hh[0], hh[1], hh[2], hh[3]);
                st16(ahi + A_BYTES, tile_off(row, c, KC), ll[0], ll[1], ll[2], ll[3]);
            }
            fence_async_smem();
            mb_arrive(&full_a[s]);
        }
    } else if (warp == 8) {
        // ---- TMA producer for the packed G' blobs ----
        int issued = 0;
        for (int kb = kb0; kb < nkb; ++kb) {
            const int s = (kb - kb0) % kBStages, u = (kb - kb0) / kBStages;
            if (u > 0 && !waitw(&empty[s], (u - 1) & 1, abort)) break;
            if (lane == 0) {
                mb_expect_tx(&full_b[s], (uint32_t)BLOB);
                tma_bulk(sm + s * STAGE + B_OFF, blob + ((int64_t)pass * nkb + kb) * SLOT, (uint32_t)BLOB, &full_b[s]);
            }
            __syncwarp();
            issued = kb - kb0 + 1;
        }
        for (int q = issued - kBStages < 0 ? 0 : issued - kBStages; q < issued; ++q) {
            volatile int no_abort = 0;
            waitw(&full_b[q % kBStages], (q / kBStages) & 1, &no_abort);
        }
    } else if (warp == 9) {
        // ---- MMA issuer ----
        const uint32_t idesc = idesc_f16(128, NP, BF);
        const uint32_t sbo = KC * 128;
        for (int kb = kb0; kb < nkb; ++kb) {
            const int s = (kb - kb0) % kBStages, u = (kb - kb0) / kBStages;
            if (!waitw(&full_a[s], u & 1, abort)) break;
            if (!waitw(&full_b[s], u & 1, abort)) break;
            tc_after();
            if (lane == 0) {
                const uint32_t st = su32(sm + s * STAGE);
                const uint32_t bhi = st + B_OFF + kHdr, blo = bhi + B_BYTES;
#pragma unroll
                for (int mt = 0; mt < kBMT; ++mt) {
                    const uint32_t ahi = st + (mt * 2) * A_BYTES, alo = ahi + A_BYTES;
                    const uint32_t d = tmem + mt * 256;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint32_t o = kk * 256;
                        umma(d, sdesc(ahi + o, 128, sbo), sdesc(bhi + o, 128, sbo), idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
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
    if (t < 256) {
        const bool ok = waitw(accf, 0, abort);
        tc_after();
        const int mt = t >> 7;
        const int i = base + t;
        // X_i[m] table in the (now idle) stage buffers, xt[m * 256 + t], when it fits;
        // otherwise every column recomputes its phase
        float2 *xt = reinterpret_cast<float2 *>(sm);
        const bool table = (kmax + 1) * 256 * (int)sizeof(float2) <= kBStages * STAGE;
        const uint32_t ux = pu[i < n ? i : 0].x;
        if (table)
            for (int m = 0; m <= kmax; ++m) {
                float cs, sn;
                phase((uint32_t)m * ux, cs, sn);
                xt[m * 256 + t] = make_float2(cs, sn);
            }
        float fx = 0.f, fy = 0.f, fz = 0.f, ph = 0.f;
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll 1
        for (int c0 = 0; c0 < NP; c0 += 16) {
            float v[16];
            tm_ld16(tmem + lanes + mt * 256 + c0, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int d = coldesc[c0 + jj];
                if (d & (1 << 12)) continue;
                const int m = d & 0xff, kind = (d >> 8) & 3, blk = (d >> 10) & 3;
                float2 x;
                if (table) x = xt[m * 256 + t];
                else phase((uint32_t)m * ux, x.x, x.y);
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
        if (ok && i < n)
            reinterpret_cast<float4 *>(bpart)[(int64_t)pass * n + i] = make_float4(fx, fy, fz, ph);
    }
    if (t == 0 && *abort) atomicOr(status, kStTimeout);
    tc_before();
    __syncthreads();
    tc_after();
    if (warp == 0) tm_dealloc(tmem, 512);
}

// Sum the passes (fixed order) into the sorted reciprocal forces and potentials.
__global__ void k_bs_reduce(int64_t n, int npass, const float *__restrict__ bpart,
                            const double4_32a *__restrict__ pg, const float *__restrict__ gscale,
                            double L, double *__restrict__ f, double *__restrict__ phi)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double sc = (double)gscale[0];
    const double qf = pg[s].w * (2.0 * kPi / L) * sc;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int ps = 0; ps < npass; ++ps) {
        const float4 v = reinterpret_cast<const float4 *>(bpart)[(int64_t)ps * n + s];
        a[0] += v.x; a[1] += v.y; a[2] += v.z; a[3] += v.w;
    }
    f[3 * s + 0] = qf * a[0];
    f[3 * s + 1] = qf * a[1];
    f[3 * s + 2] = qf * a[2];
    phi[s] = sc * a[3];
}

// ---- plan-side state ----------------------------------------------------------------------

struct TcState {
    int nf = 0;           // forward columns (2 k_max + 1 rounded up to 16)
    int sa = 0, sx = 0, sp = 0;   // forward ring depths: phases, columns, coordinates
    int kch = kFChunk;    // forward stages per TMEM accumulation
    size_t fsmem = 0;     // forward dynamic shared memory
    int ntiles = 0;       // tiles of 64 forward rows (reduction grid)
    int ngroups = 0;      // forward groups of 128 rows
    int nvg = 0;          // forward virtual groups (group, column pass)
    int maxp = 0;         // forward partial sums per virtual group (bound)
    std::vector<int4> vgs_h;      // (first row, pass, columns, 0) per virtual group
    std::vector<int2> gvg_h;      // (first virtual group, passes) per group
    int4 *vgs = nullptr;
    int2 *gvg = nullptr;
    int ncol = 0;         // back-scatter columns 3 (2 k_max + 1)
    int npass = 0, np = 0, nkb = 0;
    int kb0[4] = {0, 0, 0, 0};     // back-scatter: first K block of every pass
    float *dpart = nullptr;        // [nvg][maxp][128 columns][256]
    uint2 *yz = nullptr;           // [stages * 32] (u_y, u_z)
    unsigned char *bblob = nullptr; // [stages][hi + lo] forward B operand
    int nstg = 0;                  // 32-particle stages (capacity)
    float *gmat = nullptr;         // [ncol][2R]
    int *gmax = nullptr;
    float *gscale = nullptr;
    unsigned char *blob = nullptr; // [npass][nkb][hdr + 2 * np * kBK * 2]
    float *bpart = nullptr;        // [npass][n][4]
};

constexpr size_t kSmemMax = 232448;   // opt-in shared memory per block (227 KB)
constexpr int kTmemCols = 512;

size_t fwd_bstage(int nf) { return (size_t)2 * nf * kFK * 2; }

// Forward ring depths within the shared-memory limit: phase tiles 32 KB, column tiles 16 KB.
void fwd_config(TcState &s)
{
    const size_t p_stage = (size_t)2 * 256 * kFK * 2, x_stage = (size_t)2 * 128 * kFK * 2;
    s.sp = 8;
    s.sa = 4;
    s.sx = 5;
    auto total = [&](int sa, int sx) {
        return sa * p_stage + sx * x_stage + (size_t)s.sp * kFK * 8 +
               (size_t)(2 * sa + 2 * sx + 2 * s.sp + 3) * 8 + 64;
    };
    while (s.sx > 2 && total(s.sa, s.sx) > kSmemMax) --s.sx;
    while (s.sa > 2 && total(s.sa, s.sx) > kSmemMax) --s.sa;
    s.fsmem = total(s.sa, s.sx);
}

int fwd_ctas(const Plan &p, int64_t W);

void tc_shape(const Plan &p, int64_t n, TcState &s)
{
    s.nf = 16 * ((2 * p.kmax + 1 + 15) / 16);
    fwd_config(s);
    s.ntiles = (p.R + 63) / 64;
    s.ngroups = (p.R + 127) / 128;
    // virtual groups: a group of 128 forward rows needs the columns |m_x| <= n_x,max of its
    // first row (forward order = reverse row order), in passes of at most 128
    s.vgs_h.clear();
    s.gvg_h.clear();
    for (int g = 0; g < s.ngroups; ++g) {
        const int fr0 = g * 128;
        const int nx = p.rows_h[p.R - 1 - fr0].nxmax;
        int nc = 16 * ((2 * nx + 1 + 15) / 16);
        if (nc > s.nf) nc = s.nf;
        const int passes = (nc + 127) / 128;
        s.gvg_h.push_back(make_int2((int)s.vgs_h.size(), passes));
        for (int cp = 0; cp < passes; ++cp)
            s.vgs_h.push_back(make_int4(fr0, cp, std::min(128, nc - 128 * cp), 0));
    }
    s.nvg = (int)s.vgs_h.size();
    s.nstg = (int)((n + kFK - 1) / kFK);
    // pieces per virtual group: a group's items meet at most G / nvg + 2 CTAs (G for the
    // largest particle count the state holds)
    s.maxp = fwd_ctas(p, (int64_t)s.nvg * s.nstg) / s.nvg + 2;
    s.ncol = 3 * (2 * p.kmax + 1);
    s.npass = (s.ncol + kPassMax - 1) / kPassMax;
    s.np = bs_pass_cols(s.ncol, 0);         // the widest pass: slot stride of the packed blobs
    s.nkb = (2 * p.R + kBK - 1) / kBK;
    // rows run in order of increasing n_x,max; pass q starts at the K block holding the first
    // row that reaches the smallest m of its columns
    for (int q = 0; q < s.npass && q < 4; ++q) {
        const int mlo = bs_col(q * kPassMax).m;
        int r = 0;
        while (r < p.R && p.rows_h[r].nxmax < mlo) ++r;
        s.kb0[q] = (r < p.R ? r : p.R - 1) / (kBK / 2);
    }
}

size_t bs_blob(int np) { return kHdr + 2 * (size_t)np * kBK * 2; }
size_t bs_smem(int np)
{
    const size_t stage = (size_t)kBMT * 2 * 128 * kBK * 2 + bs_blob(np);
    return kBStages * stage + 128 + 4 * (size_t)np;
}

// CTAs of the forward product: one per SM, but at least kFMinItems (virtual group, stage)
// items each, so that a small system (a serving request of a few thousand particles) leaves
// most SMs to the products of other requests instead of spreading a few items over all of
// them (every CTA holds 210 KB of shared memory for its whole life).  Large systems run up to
// four waves of CTAs, so that a CTA's segment holds at most about kFSegItems items: the FP32
// running sum in tensor memory takes one addition per 128-particle chunk of the segment, and
// its rounding grows with their number (measured at 2,097,152 ions: S(k) error 4.4e-7 with
// one wave, 3.3e-7 with four, forward time unchanged).
constexpr int64_t kFMinItems = 16;
constexpr int64_t kFSegItems = 4096;
int fwd_ctas(const Plan &p, int64_t W)
{
    const int64_t waves = std::max<int64_t>(1, std::min<int64_t>(4, W / ((int64_t)p.num_sms * kFSegItems)));
    const int64_t g = (W + kFMinItems - 1) / kFMinItems;
    return (int)std::max<int64_t>(1, std::min<int64_t>(waves * p.num_sms, g));
}

template <bool BF>
cudaError_t launch_fwd(Plan &p, int nst_all, TcState &s, cudaStream_t st)
{
    cudaError_t e = smem_optin((const void *)k_fwd_tc<BF>);
    if (e != cudaSuccess) return e;
    const int64_t W = (int64_t)s.nvg * nst_all;
    const int G = fwd_ctas(p, W);
    k_fwd_tc<BF><<<G, kFThreads, s.fsmem, st>>>(
        p.R, s.nf, nst_all, W, s.maxp, s.sa, s.sx, s.sp, s.kch, s.vgs, p.rows_d, p.fperm_d, s.yz,
        s.bblob, s.dpart, p.d_status);
    return cudaGetLastError();
}

template <bool BF>
cudaError_t launch_bf(Plan &p, int64_t n, cudaStream_t st)
{
    TcState &s = *static_cast<TcState *>(p.tc);
    Workspace &ws = p.ws;
    cudaError_t e;
    prof_mark(p, kEvRecipStart, st);
    const int nst_all = (int)((n + kFK - 1) / kFK);
    e = launch_fwd<BF>(p, nst_all, s, st);
    if (e != cudaSuccess) return e;
    prof_mark(p, kEvFwdEnd, st);
    if ((e = cudaMemsetAsync(s.gmax, 0, sizeof(int), st)) != cudaSuccess) return e;
    {
        const int64_t W = (int64_t)s.nvg * nst_all;
        const int G = fwd_ctas(p, W);
        k_sreduce_tc<<<dim3(s.ntiles, p.kmax + 1), 64, 0, st>>>(
            nst_all, W, G, s.maxp, s.gvg, s.ntiles, p.R, p.kmax, s.nf, p.rows_d, p.fperm_d,
            s.dpart, p.g_d, p.S_d, p.e_recip_part, s.gmat, s.gmax);
    }
    k_bpack<BF><<<dim3(s.nkb, s.npass), 256, 0, st>>>(p.R, s.ncol, s.np, s.nkb, p.rows_d, s.gmat,
                                                      s.gmax, s.gscale, s.blob);
    prof_mark(p, kEvCoefEnd, st);
    const size_t bs = bs_smem(s.np);
    if ((e = smem_optin((const void *)k_bs_tc<BF>)) != cudaSuccess) return e;
    const int ptiles = (int)((n + kBMT * 128 - 1) / (kBMT * 128));
    prof_mark(p, kEvBsStart, st);
    k_bs_tc<BF><<<dim3(ptiles, s.npass), kBThreads, bs, st>>>(
        (int)n, p.R, p.kmax, s.ncol, s.np, s.nkb, make_int4(s.kb0[0], s.kb0[1], s.kb0[2], s.kb0[3]),
        ws.pu, s.blob, s.bpart, p.d_status);
    prof_mark(p, kEvBsEnd, st);
    p.prof_bs = p.prof;
    k_bs_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, s.npass, s.bpart, ws.pg, s.gscale,
                                                            p.L, ws.f_recip, ws.phi_recip);
    prof_mark(p, kEvBackEnd, st);
    p.launches += 5;
    return cudaGetLastError();
}

}  // namespace

int recip_tc_energy_parts(const Plan &p) { return ((p.R + 63) / 64) * (p.kmax + 1); }

size_t recip_tc_bytes(const Plan &p, int64_t n)
{
    TcState s;
    tc_shape(p, n, s);
    size_t b = 0;
    b += (size_t)s.nvg * s.maxp * 128 * 256 * sizeof(float);
    b += (size_t)s.nvg * sizeof(int4) + (size_t)s.ngroups * sizeof(int2);
    b += (size_t)s.nstg * (fwd_bstage(s.nf) + kFK * sizeof(uint2));
    b += (size_t)2 * p.R * s.ncol * sizeof(float);
    b += (size_t)s.npass * s.nkb * bs_blob(s.np);
    b += (size_t)s.npass * n * 4 * sizeof(float);
    return b + 1024;
}

cudaError_t alloc_recip_tc(Plan &p, int64_t n)
{
    free_recip_tc(p);
    TcState *s = new TcState();
    tc_shape(p, n, *s);
    p.tc = s;
    cudaStream_t st = p.side_stream;
    cudaError_t e;
    if ((e = pool_alloc((void **)&s->dpart, (size_t)s->nvg * s->maxp * 128 * 256 * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->vgs, (size_t)s->nvg * sizeof(int4), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gvg, (size_t)s->ngroups * sizeof(int2), st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(s->vgs, s->vgs_h.data(), (size_t)s->nvg * sizeof(int4), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(s->gvg, s->gvg_h.data(), (size_t)s->ngroups * sizeof(int2), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gmat, (size_t)2 * p.R * s->ncol * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->yz, (size_t)s->nstg * kFK * sizeof(uint2), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->bblob, (size_t)s->nstg * fwd_bstage(s->nf), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gmax, 64, st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->gscale, 64, st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->blob, (size_t)s->npass * s->nkb * bs_blob(s->np), st)) != cudaSuccess) return e;
    if ((e = pool_alloc((void **)&s->bpart, (size_t)s->npass * n * 4 * sizeof(float), st)) != cudaSuccess) return e;
    return cudaSuccess;
}

void free_recip_tc(Plan &p)
{
    TcState *s = static_cast<TcState *>(p.tc);
    if (!s) return;
    cudaStream_t st = p.side_stream;
    pool_free(s->dpart, st); pool_free(s->gmat, st); pool_free(s->gmax, st);
    pool_free(s->vgs, st); pool_free(s->gvg, st);
    pool_free(s->yz, st); pool_free(s->bblob, st);
    pool_free(s->gscale, st); pool_free(s->blob, st); pool_free(s->bpart, st);
    delete s;
    p.tc = nullptr;
}

cudaError_t launch_recip_tc_operands(Plan &p, int64_t n, cudaStream_t st)
{
    if (!p.tc) return cudaErrorInvalidValue;
    TcState &s = *static_cast<TcState *>(p.tc);
    const int nst_all = (int)((n + kFK - 1) / kFK);
    if (p.precision == EWALD_MIXED_BF16)
        k_xgen<true><<<nst_all, 256, 0, st>>>((int)n, p.kmax, s.nf, p.ws.pu, s.yz, s.bblob);
    else
        k_xgen<false><<<nst_all, 256, 0, st>>>((int)n, p.kmax, s.nf, p.ws.pu, s.yz, s.bblob);
    p.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_recip_tc(Plan &p, int64_t n, cudaStream_t st)
{
    if (!p.tc) return cudaErrorInvalidValue;
    if (p.precision == EWALD_MIXED_BF16) return launch_bf<true>(p, n, st);
    return launch_bf<false>(p, n, st);
}

}  // namespace ew
