// Integer cell binning (hot-path steps a1-a3): periodic wrap, cell keys, a stable
// counting sort by cell, cell offsets, and packing of the sorted particles.
//
// The paper's short-range part runs as a "local PairLoop" that only visits pairs closer
// than r_c through cell-based looping code (Section 2.2; Section 3.2.1).  Here the cells
// are a regular grid of nc^3 cubes of side L / nc >= r_c / w; particles are sorted by cell
// key (c_z nc + c_y) nc + c_x so that every cell, and every row of cells along x, is a
// contiguous range of the sorted arrays.  The sort is a two-pass counting sort over
// `nb` contiguous chunks of the input: per-chunk histograms, a column scan over chunks, a
// scan over cells, and an in-order scatter per chunk; equal keys keep their input order, so
// the result is exactly determined by the input (bit-exact integer work).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace ew {
namespace {

__device__ __forceinline__ double wrap_box(double x, double L)
{
    // x - L floor(x / L), with explicit rounding steps (no fused multiply-add) so that the
    // result is reproducible on any IEEE machine; a result equal to L maps to 0.  A position
    // already in [0, L) gives the same result without the FP64 division: x / L rounds to at
    // most 1 - 2^-53 there, so the floor is 0 and the result is x - 0 (+0 for x = -0).
    if (x >= 0.0 && x < L) return __dadd_rn(x, 0.0);
    double w = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    return (w >= L) ? 0.0 : w;
}

__device__ __forceinline__ int cell_of(double w, double inv_side, int nc)
{
    int c = (int)__dmul_rn(w, inv_side);
    return c < nc - 1 ? c : nc - 1;
}

// a1: wrap + key + per-chunk histogram; finiteness flag; per-block charge sums.
__global__ void k_keys(int64_t n, const double *__restrict__ pos, const double *__restrict__ q,
                       double L, double inv_side, int nc, int ncells, int64_t chunk,
                       int *__restrict__ key, int *__restrict__ hist, double *__restrict__ qpart,
                       int *__restrict__ status)
{
    __shared__ double red[3][32];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double qs = 0.0, qa = 0.0, q2 = 0.0;
    if (i < n) {
        double x = pos[3 * i + 0], y = pos[3 * i + 1], z = pos[3 * i + 2], qi = q[i];
        bool fin = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qi);
        if (!fin) {
            atomicOr(status, kStNonFinite);
            x = y = z = 0.0;
            qi = 0.0;
        }
        int cx = cell_of(wrap_box(x, L), inv_side, nc);
        int cy = cell_of(wrap_box(y, L), inv_side, nc);
        int cz = cell_of(wrap_box(z, L), inv_side, nc);
        int k = (cz * nc + cy) * nc + cx;
        key[i] = k;
        atomicAdd(&hist[(i / chunk) * (int64_t)ncells + k], 1);
        qs = qi;
        qa = fabs(qi);
        q2 = qi * qi;
    }
    // fixed-order block reduction (shuffle tree, then warp 0 over the warp sums)
    for (int o = 16; o > 0; o >>= 1) {
        qs += __shfl_down_sync(0xffffffffu, qs, o);
        qa += __shfl_down_sync(0xffffffffu, qa, o);
        q2 += __shfl_down_sync(0xffffffffu, q2, o);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[0][wid] = qs; red[1][wid] = qa; red[2][wid] = q2; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        qs = lane < nw ? red[0][lane] : 0.0;
        qa = lane < nw ? red[1][lane] : 0.0;
        q2 = lane < nw ? red[2][lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            qs += __shfl_down_sync(0xffffffffu, qs, o);
            qa += __shfl_down_sync(0xffffffffu, qa, o);
            q2 += __shfl_down_sync(0xffffffffu, q2, o);
        }
        if (lane == 0) {
            qpart[3 * blockIdx.x + 0] = qs;
            qpart[3 * blockIdx.x + 1] = qa;
            qpart[3 * blockIdx.x + 2] = q2;
        }
    }
}

// a2 (part): exclusive prefix over chunks, per cell, in place; cell totals.  The chunk
// counts of a cell are read 16 at a time so that the loads overlap.
__global__ void k_colscan(int nb, int ncells, int *__restrict__ hist, int *__restrict__ total)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int run = 0;
    for (int b0 = 0; b0 < nb; b0 += 16) {
        int h[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) h[u] = b0 + u < nb ? hist[(int64_t)(b0 + u) * ncells + c] : 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (b0 + u < nb) hist[(int64_t)(b0 + u) * ncells + c] = run;
            run += h[u];
        }
    }
    total[c] = run;
}

// Exclusive scan of cnt[0..m) into out[0..m] (out[m] = total), one block of 1024 threads.
// Every thread scans a contiguous slice serially; slice sums are scanned in shared memory.
__global__ void k_scan1(int m, const int *__restrict__ cnt, int *__restrict__ out)
{
    __shared__ int part[1024];
    int t = threadIdx.x;
    int per = (m + blockDim.x - 1) / blockDim.x;
    int b = t * per, e = min(m, b + per);
    int s = 0;
    for (int c = b; c < e; ++c) s += cnt[c];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;  // exclusive prefix of this slice
    for (int c = b; c < e; ++c) {
        int v = cnt[c];
        out[c] = run;
        run += v;
    }
    if (t == blockDim.x - 1) out[m] = part[t];
}

// a2 (part): in-order scatter of chunk b.  The whole block loads the chunk's running
// offsets per cell and the chunk's keys into shared memory; then warp 0 walks the chunk in
// input order, 32 particles at a time.  (When the offsets do not fit, the chunk's histogram
// row in global memory holds them.)
__global__ void k_scatter(int64_t n, int64_t chunk, int ncells, const int *__restrict__ key,
                          const int *__restrict__ cell_start, int *__restrict__ hist,
                          int *__restrict__ perm, int *__restrict__ key_sorted, int use_smem)
{
    extern __shared__ int sh[];
    const int b = blockIdx.x;
    const int64_t beg = (int64_t)b * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    const int cnt = (int)(end > beg ? end - beg : 0);
    int *keys = sh;                              // [chunk]
    int *row = hist + (int64_t)b * ncells;
    int *off = use_smem ? sh + chunk : row;
    // (eight cells per thread per step, so that the loads overlap)
    for (int c0 = threadIdx.x; c0 < ncells; c0 += 8 * blockDim.x) {
        int r[8], s[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * blockDim.x;
            r[u] = c < ncells ? row[c] : 0;
            s[u] = c < ncells ? cell_start[c] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = c0 + u * blockDim.x;
            if (c < ncells) off[c] = r[u] + s[u];
        }
    }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) keys[i] = key[beg + i];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const bool valid = i < cnt;
        const int k = valid ? keys[i] : -1 - lane;   // invalid lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int rank = __popc(peers & lt);
        const int leader = __ffs(peers) - 1;
        const int start = valid ? off[k] : 0;
        __syncwarp();
        if (valid) {
            const int slot = start + rank;
            perm[slot] = (int)(beg + i);
            key_sorted[slot] = k;
            if (lane == leader) off[k] = start + __popc(peers);
        }
        __syncwarp();
    }
}

// a3: pack sorted particles: wrapped global FP64 position, cell-local FP64 / FP32 positions
// (the all-pairs kernel, written only in that mode) and 32-bit fixed-point fractions of the
// box (the FP32 cell kernel's exact minimum-image displacements and the exact integer phase
// angles of the tensor-core reciprocal part).
__global__ void k_pack(int64_t n, const double *__restrict__ pos, const double *__restrict__ q,
                       const int *__restrict__ perm, const int *__restrict__ key_sorted,
                       double L, double side, int nc,
                       double4_32a *__restrict__ pg, double4_32a *__restrict__ pl64,
                       float4 *__restrict__ pl32, uint4 *__restrict__ pu)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    double x = pos[3 * (int64_t)i + 0], y = pos[3 * (int64_t)i + 1], z = pos[3 * (int64_t)i + 2];
    double qi = q[i];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qi))) { x = y = z = 0.0; qi = 0.0; }
    x = wrap_box(x, L); y = wrap_box(y, L); z = wrap_box(z, L);
    int k = key_sorted[s];
    int cx = k % nc, cy = (k / nc) % nc, cz = k / (nc * nc);
    pg[s] = make_double4_32a(x, y, z, qi);
    double lx = x - cx * side, ly = y - cy * side, lz = z - cz * side;
    const double scale = 4294967296.0 / L;
    unsigned ux = (unsigned)((unsigned long long)llrint(x * scale) & 0xffffffffull);
    if (pl64) pl64[s] = make_double4_32a(lx, ly, lz, qi);
    if (pl32) pl32[s] = make_float4((float)lx, (float)ly, (float)lz, (float)qi);
    if (pu) {
        unsigned uy = (unsigned)((unsigned long long)llrint(y * scale) & 0xffffffffull);
        unsigned uz = (unsigned)((unsigned long long)llrint(z * scale) & 0xffffffffull);
        pu[s] = make_uint4(ux, uy, uz, __float_as_uint((float)qi));
    }
}

// Tiles of up to `ts` consecutive sorted particles that never leave a row of cells (the
// targets of one warp of the cell kernel share their row, so that the warp can stage one
// union of candidate ranges per stencil row for all of them).
__global__ void k_row_tiles(int nrows, int nc, int ts, const int *__restrict__ cell_start,
                            int *__restrict__ tcount)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int cnt = cell_start[(r + 1) * nc] - cell_start[r * nc];
    tcount[r] = (cnt + ts - 1) / ts;
}

__global__ void k_emit_tiles(int nrows, int nc, int ts, const int *__restrict__ cell_start,
                             const int *__restrict__ toff, int2 *__restrict__ tiles)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int b = cell_start[r * nc];
    int o = toff[r], e = toff[r + 1];
    for (int t = o; t < e; ++t) tiles[t] = make_int2(r, b + ts * (t - o));
}

}  // namespace

cudaError_t launch_binning(Plan &p, int64_t n, const double *pos, const double *q,
                           cudaStream_t st)
{
    Workspace &ws = p.ws;
    const int nb = ws.nb;
    const int64_t chunk = (n + nb - 1) / nb;
    cudaError_t e;
    e = cudaMemsetAsync(ws.hist, 0, sizeof(int) * (size_t)nb * p.ncells, st);
    if (e != cudaSuccess) return e;
    const int tb = 256;
    const int qblocks = (int)((n + tb - 1) / tb);
    k_keys<<<qblocks, tb, 0, st>>>(n, pos, q, p.L, (double)p.nc / p.L, p.nc, p.ncells, chunk,
                                   ws.key, ws.hist, ws.qpart, p.d_status);
    k_colscan<<<(p.ncells + 255) / 256, 256, 0, st>>>(nb, p.ncells, ws.hist, ws.cell_total);
    k_scan1<<<1, 1024, 0, st>>>(p.ncells, ws.cell_total, ws.cell_start);
    const size_t key_bytes = sizeof(int) * (size_t)chunk;
    const int use_smem = key_bytes + sizeof(int) * (size_t)p.ncells <= 200 * 1024;
    size_t smem = key_bytes + (use_smem ? sizeof(int) * (size_t)p.ncells : 0);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_scatter<<<nb, 256, smem, st>>>(n, chunk, p.ncells, ws.key, ws.cell_start, ws.hist, ws.perm,
                                     ws.key_sorted, use_smem);
    const bool need64 = p.precision == EWALD_FP64;
    k_pack<<<(int)((n + 255) / 256), 256, 0, st>>>(n, pos, q, ws.perm, ws.key_sorted, p.L,
                                                   p.cell_side, p.nc, ws.pg,
                                                   (need64 && p.w == 0) ? ws.pl64 : nullptr,
                                                   (!need64 && p.w == 0) ? ws.pl32 : nullptr, ws.pu);
    p.launches += 5;
    if (p.w > 0) {
        const int nrows = p.nc * p.nc;
        const int ts = real_tile_size(p);
        k_row_tiles<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p.nc, ts, ws.cell_start,
                                                         ws.tile_count);
        k_scan1<<<1, 1024, 0, st>>>(nrows, ws.tile_count, ws.tile_off);
        k_emit_tiles<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p.nc, ts, ws.cell_start,
                                                          ws.tile_off, ws.tiles);
        p.launches += 3;
    }
    return cudaGetLastError();
}

}  // namespace ew
