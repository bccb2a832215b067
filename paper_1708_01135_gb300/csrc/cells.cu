// Integer cell binning (hot-path steps a1-a3): periodic wrap, cell keys, a stable
// counting sort by cell, cell offsets, and packing of the sorted particles.
//
// The paper's short-range part runs as a "local PairLoop" that only visits pairs closer
// than r_c through cell-based looping code (Section 2.2; Section 3.2.1).  Here the cells
// are a regular grid of nc^3 cubes of side L / nc >= r_c / w; particles are sorted by cell
// key (c_z nc + c_y) nc + c_x so that every cell, and every row of cells along x, is a
// contiguous range of the sorted arrays.  The sort runs in two levels, each a stable
// counting sort, so that no histogram spans all cells:
//   1. by row of cells (c_z nc + c_y) over `nb` contiguous chunks of the input: per-chunk
//      row histograms, a column scan over chunks, a scan over rows, and an in-order scatter
//      per chunk;
//   2. inside every row, by c_x: one block per row counts its cells, scans them (the cell
//      offsets) and places the row's particles in the order level 1 left them; where the
//      cell kernel cuts its ranges to x windows, every cell is then ordered by x
//      (fixed-point fraction, k_rowsort).
// Equal keys keep their input order, so the result is exactly determined by the input
// (bit-exact integer work).
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

// a1: wrap + key + per-chunk histogram of rows; finiteness flag; per-block charge sums.
__global__ void k_keys(int64_t n, const double *__restrict__ pos, const double *__restrict__ q,
                       double L, double inv_side, int nc, int nrows, int64_t chunk,
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
        atomicAdd(&hist[(i / chunk) * (int64_t)nrows + (cz * nc + cy)], 1);
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

// a2 (level 1): in-order scatter of chunk b by row.  The whole block loads the chunk's
// running offsets per row and the chunk's keys into shared memory; then warp 0 walks the
// chunk in input order, 32 particles at a time.  (When the offsets do not fit, the chunk's
// histogram row in global memory holds them.)
__global__ void k_scatter(int64_t n, int64_t chunk, int nrows, int nc, const int *__restrict__ key,
                          const int *__restrict__ row_start, int *__restrict__ hist,
                          int *__restrict__ perm1, int *__restrict__ key1, int use_smem)
{
    const int ncells = nrows;
    const int *__restrict__ cell_start = row_start;
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
        const int key_i = valid ? keys[i] : 0;
        const int k = valid ? key_i / nc : -1 - lane;   // the row; invalid lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int rank = __popc(peers & lt);
        const int leader = __ffs(peers) - 1;
        const int start = valid ? off[k] : 0;
        __syncwarp();
        if (valid) {
            const int slot = start + rank;
            perm1[slot] = (int)(beg + i);
            key1[slot] = key_i;
            if (lane == leader) off[k] = start + __popc(peers);
        }
        __syncwarp();
    }
}

// a3: pack sorted particle s (caller index i, cell key k): wrapped global FP64 position,
// cell-local FP64 / FP32 positions (the all-pairs kernel, written only in that mode) and
// 32-bit fixed-point fractions of the box (the FP32 cell kernel's exact minimum-image
// displacements and the exact integer phase angles of the tensor-core reciprocal part).
__device__ __forceinline__ void pack_one(int64_t s, int i, int k, const double *__restrict__ pos,
                                         const double *__restrict__ q, double L, double side,
                                         int nc, double4_32a *__restrict__ pg,
                                         double4_32a *__restrict__ pl64,
                                         float4 *__restrict__ pl32, uint4 *__restrict__ pu)
{
    double x = pos[3 * (int64_t)i + 0], y = pos[3 * (int64_t)i + 1], z = pos[3 * (int64_t)i + 2];
    double qi = q[i];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(qi))) { x = y = z = 0.0; qi = 0.0; }
    x = wrap_box(x, L); y = wrap_box(y, L); z = wrap_box(z, L);
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

// Exclusive scans of the particles per row of cells (row_start[0..nrows]) and, with ts > 0,
// of the warp tiles per row, ceil(count / ts) (tile_off[0..nrows]): the targets of one warp
// of the cell kernel never leave a row, so that the warp can stage one union of candidate
// ranges per stencil row for all of them.  One block of 1024 threads: every thread scans a
// contiguous slice serially; slice sums are scanned in shared memory.
__global__ void k_scan_rows(int nrows, int ts, const int *__restrict__ cnt,
                            int *__restrict__ row_start, int *__restrict__ tile_off,
                            int *__restrict__ unordered)
{
    __shared__ int part[2][1024];
    const int t = threadIdx.x;
    if (t == 0) *unordered = 0;      // (k_rowsort sets it for a cell it cannot order)
    const int per = (nrows + blockDim.x - 1) / blockDim.x;
    const int b = t * per, e = min(nrows, b + per);
    int s0 = 0, s1 = 0;
    for (int r = b; r < e; ++r) {
        const int v = cnt[r];
        s0 += v;
        s1 += ts > 0 ? (v + ts - 1) / ts : 0;
    }
    part[0][t] = s0;
    part[1][t] = s1;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v0 = t >= o ? part[0][t - o] : 0, v1 = t >= o ? part[1][t - o] : 0;
        __syncthreads();
        part[0][t] += v0;
        part[1][t] += v1;
        __syncthreads();
    }
    int run0 = part[0][t] - s0, run1 = part[1][t] - s1;   // exclusive prefixes of the slice
    for (int r = b; r < e; ++r) {
        const int v = cnt[r];
        row_start[r] = run0;
        run0 += v;
        if (ts > 0) {
            tile_off[r] = run1;
            run1 += (v + ts - 1) / ts;
        }
    }
    if (t == blockDim.x - 1) {
        row_start[nrows] = part[0][t];
        if (ts > 0) tile_off[nrows] = part[1][t];
    }
}

// Cells of more particles than this keep the order of level 2 (the x order below costs a
// pass over the cell per particle).
constexpr int kXOrderMax = 256;

// a2 (level 2) and a3: row r of cells (particles [row_start[r], row_start[r+1]) in level-1
// order): counts per cell, the cell offsets cell_start[r nc .. r nc + nc - 1], the in-order
// placement of the row's particles by cell (warp 0), then the packing of the row's sorted
// particles and, with tiles, the row's warp tiles (all threads).  One block per row.
// With xorder (the cell kernel's x windows, use_xwin) the particles of every cell are ordered
// by x before they are packed: by the 32-bit fixed-point fraction that the packed record
// holds, taken relative to the cell's centre (so a fraction that rounds to 2^32 next to
// x = L stays at the end of the last cell), equal fractions in level-2 order.  The
// real-space kernel cuts each target's range at its own x window with this order.  A cell
// of more than kXOrderMax particles keeps its level-2 order and sets *unordered, which
// turns the cut off.
__global__ void k_rowsort(int nrows, int nc, int64_t n, const int *__restrict__ row_start,
                          int *__restrict__ perm1, int *__restrict__ key1,
                          int *__restrict__ perm, int *__restrict__ key_sorted,
                          int *__restrict__ cell_start, const double *__restrict__ pos,
                          const double *__restrict__ q, double L, double side,
                          double4_32a *__restrict__ pg, double4_32a *__restrict__ pl64,
                          float4 *__restrict__ pl32, uint4 *__restrict__ pu, int ts,
                          const int *__restrict__ tile_off, int2 *__restrict__ tiles,
                          int xorder, int *__restrict__ unordered)
{
    __shared__ int off[kMaxCellsPerSide];
    const int r = blockIdx.x;
    const int b = row_start[r], e = row_start[r + 1];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) off[c] = 0;
    __syncthreads();
    for (int j = b + threadIdx.x; j < e; j += blockDim.x) atomicAdd(&off[key1[j] % nc], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = b;
        for (int c = 0; c < nc; ++c) {
            const int v = off[c];
            off[c] = run;
            cell_start[r * nc + c] = run;
            run += v;
        }
        if (r == nrows - 1) cell_start[nrows * nc] = (int)n;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned lt = (1u << lane) - 1u;
        for (int base = b; base < e; base += 32) {
            const int j = base + lane;
            const bool valid = j < e;
            const int key_j = valid ? key1[j] : 0;
            const int cx = valid ? key_j % nc : -1 - lane;
            const unsigned peers = __match_any_sync(0xffffffffu, cx);
            const int rank = __popc(peers & lt);
            const int leader = __ffs(peers) - 1;
            const int start = valid ? off[cx] : 0;
            __syncwarp();
            if (valid) {
                const int slot = start + rank;
                perm[slot] = perm1[j];
                key_sorted[slot] = key_j;
                if (lane == leader) off[cx] = start + __popc(peers);
            }
            __syncwarp();
        }
    }
    // (the block's own global writes are visible to the block after the barrier)
    __syncthreads();
    if (xorder) {
        // x order inside every cell; perm1 and key1 of the row (read only by this block, and
        // no longer needed) hold the level-2 order and the sort keys
        const double scale = 4294967296.0 / L;
        for (int s = b + threadIdx.x; s < e; s += blockDim.x) {
            const int i = perm[s];
            double x = pos[3 * (int64_t)i + 0];
            const double y = pos[3 * (int64_t)i + 1], z = pos[3 * (int64_t)i + 2];
            if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(q[i]))) x = 0.0;
            x = wrap_box(x, L);
            const unsigned ux = (unsigned)((unsigned long long)llrint(x * scale) & 0xffffffffull);
            const int c = key_sorted[s] % nc;
            const unsigned uc =
                (unsigned)((unsigned long long)llrint(((double)c + 0.5) * side * scale) & 0xffffffffull);
            key1[s] = (int)(ux - uc);
            perm1[s] = i;
        }
        __syncthreads();
        for (int s = b + threadIdx.x; s < e; s += blockDim.x) {
            const int c = key_sorted[s] % nc;
            const int cb = cell_start[r * nc + c];
            const int ce = c + 1 < nc ? cell_start[r * nc + c + 1] : e;
            if (ce - cb > kXOrderMax) {
                *unordered = 1;                  // (perm[s] is still perm1[s])
                continue;
            }
            const int v = key1[s];
            int rank = 0;
            for (int t = cb; t < ce; ++t) {
                const int u = key1[t];
                rank += (u < v) || (u == v && t < s);
            }
            perm[cb + rank] = perm1[s];
        }
        __syncthreads();
    }
    for (int s = b + threadIdx.x; s < e; s += blockDim.x)
        pack_one(s, perm[s], key_sorted[s], pos, q, L, side, nc, pg, pl64, pl32, pu);
    if (tiles) {
        const int o = tile_off[r], oe = tile_off[r + 1];
        for (int t = o + threadIdx.x; t < oe; t += blockDim.x) tiles[t] = make_int2(r, b + ts * (t - o));
    }
}

}  // namespace

cudaError_t launch_binning(Plan &p, int64_t n, const double *pos, const double *q,
                           cudaStream_t st)
{
    Workspace &ws = p.ws;
    const int nb = ws.nb;
    const int64_t chunk = (n + nb - 1) / nb;
    cudaError_t e;
    const int nrows = p.nc * p.nc;
    e = cudaMemsetAsync(ws.hist, 0, sizeof(int) * (size_t)nb * nrows, st);
    if (e != cudaSuccess) return e;
    const int tb = 256;
    const int qblocks = (int)((n + tb - 1) / tb);
    k_keys<<<qblocks, tb, 0, st>>>(n, pos, q, p.L, (double)p.nc / p.L, p.nc, nrows, chunk,
                                   ws.key, ws.hist, ws.qpart, p.d_status);
    k_colscan<<<(nrows + 255) / 256, 256, 0, st>>>(nb, nrows, ws.hist, ws.cell_total);
    const int ts = p.w > 0 ? real_tile_size(p) : 0;
    k_scan_rows<<<1, 1024, 0, st>>>(nrows, ts, ws.cell_total, ws.row_start, ws.tile_off,
                                    ws.unordered);
    const size_t key_bytes = sizeof(int) * (size_t)chunk;
    const int use_smem = key_bytes + sizeof(int) * (size_t)nrows <= 200 * 1024;
    size_t smem = key_bytes + (use_smem ? sizeof(int) * (size_t)nrows : 0);
    if (smem > 48 * 1024) {
        e = smem_optin((const void *)k_scatter);
        if (e != cudaSuccess) return e;
    }
    k_scatter<<<nb, 256, smem, st>>>(n, chunk, nrows, p.nc, ws.key, ws.row_start, ws.hist,
                                     ws.perm1, ws.key1, use_smem);
    const bool need64 = p.precision == EWALD_FP64;
    k_rowsort<<<nrows, 128, 0, st>>>(nrows, p.nc, n, ws.row_start, ws.perm1, ws.key1, ws.perm,
                                     ws.key_sorted, ws.cell_start, pos, q, p.L, p.cell_side,
                                     ws.pg, (need64 && p.w == 0) ? ws.pl64 : nullptr,
                                     (!need64 && p.w == 0) ? ws.pl32 : nullptr, ws.pu, ts,
                                     ws.tile_off, p.w > 0 ? ws.tiles : nullptr, use_xwin(p),
                                     ws.unordered);
    p.launches += 5;
    return cudaGetLastError();
}

}  // namespace ew
