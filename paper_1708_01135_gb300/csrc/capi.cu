// C ABI of libewald.so: plans, the per-call pipeline, the self/total step (a9), the tuner.
//
// One evaluation (ewald_compute_async) on the caller's stream:
//   a1-a3  binning: wrap, cell keys, stable counting sort, offsets, packing   (cells.cu)
//   a5     the column operand of the forward product (tensor path), still on the caller's
//          stream, so that the forward product and the real-space kernel become ready
//          together and the forward's one-CTA-per-SM grid is placed first
//   fork:  the reciprocal branch runs on the plan's side stream
//   a4     real-space pairs                                                    (realspace.cu)
//   a5-a8  phases, S(k), energy and coefficients, back-scatter    (recip_simt.cu / recip_tc.cu)
//   join, a9: self energy -beta/sqrt(pi) sum q^2 (Section 3.2.2), energy totals, neutrality
//          check, and the sum of the force parts scattered back to the caller's order.
// Every reduction is a fixed-order tree or serial sum, so repeated calls with the same input
// give bit-identical results.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "ewald_internal.cuh"

using namespace ew;

static void cell_grid(double L, double rc, int64_t n, int &nc, int &w);


namespace ew {
namespace {

// Sum of x[0..m) by one thread block of 256 threads in a fixed order: thread t sums the
// elements t, t + 256, t + 512, ... (coalesced loads) into 4 partial sums by position modulo
// 4, combines them in order, then a fixed tree over the threads.  Every thread returns the
// total.
__device__ double block_sum_fixed(const double *__restrict__ x, int m, double *red)
{
    const int t = threadIdx.x;
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    int i = t;
    for (; i + 3 * 256 < m; i += 4 * 256) {
        p[0] += x[i];
        p[1] += x[i + 256];
        p[2] += x[i + 512];
        p[3] += x[i + 768];
    }
    for (int u = 0; i < m; i += 256, ++u) p[u] += x[i];
    double s = (p[0] + p[1]) + (p[2] + p[3]);
    red[t] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    s = red[0];
    __syncthreads();
    return s;
}

// a9: energies (one block, fixed order) and the neutrality check.
// With elj_tile (Lennard-Jones pairs on), their energy is part of energy[3] only.
__global__ void k_energy(int ntile, const double *__restrict__ e_tile, int nq,
                         const double *__restrict__ qpart, int R,
                         const double *__restrict__ e_row, double beta, int parts,
                         const double *__restrict__ elj_tile, int spme,
                         double *__restrict__ energy, int *__restrict__ status)
{
    __shared__ double red[256];
    __shared__ double qv[3][256];
    const double er = block_sum_fixed(e_tile, ntile, red);
    const double ek = block_sum_fixed(e_row, R, red);
    const double elj = elj_tile ? block_sum_fixed(elj_tile, ntile, red) : 0.0;
    // charge sums: qpart is [nq][3]
    const int t = threadIdx.x;
    double qs = 0.0, qa = 0.0, q2 = 0.0;
    for (int i = t; i < nq; i += 256) {
        qs += qpart[3 * i]; qa += qpart[3 * i + 1]; q2 += qpart[3 * i + 2];
    }
    qv[0][t] = qs; qv[1][t] = qa; qv[2][t] = q2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) {
            qv[0][t] += qv[0][t + o]; qv[1][t] += qv[1][t + o]; qv[2][t] += qv[2][t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        qs = qv[0][0]; qa = qv[1][0]; q2 = qv[2][0];
        if (fabs(qs) > 1e-10 * qa) atomicOr(status, kStNonNeutral);
        if (spme && !(qa < kSpmeMaxAbsCharge)) atomicOr(status, kStRange);
        const double e_real = (parts & EWALD_PART_REAL) ? 0.5 * er : 0.0;
        const double e_recip = (parts & EWALD_PART_RECIP) ? ek : 0.0;
        const double e_self = (parts & EWALD_PART_SELF) ? -beta / sqrt(kPi) * q2 : 0.0;
        energy[0] = e_real;
        energy[1] = e_recip;
        energy[2] = e_self;
        energy[3] = ((e_real + e_recip) + e_self) + elj;
    }
}

// Lennard-Jones types in sorted order; a type outside [0, ntypes) is replaced by 0 and
// flagged.
__global__ void k_gather_type(int64_t n, const int *__restrict__ perm, const int *__restrict__ type,
                              int ntypes, int *__restrict__ tsort, int *__restrict__ status)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int t = type[perm[s]];
    if (t < 0 || t >= ntypes) {
        atomicOr(status, kStBadType);
        t = 0;
    }
    tsort[s] = t;
}

// a9: F[perm[s]] = F_real[s] + F_recip[s] (selected parts), caller order.
// With phi_out: phi[perm[s]] = phi_real[s] + phi_recip[s] - 2 beta / sqrt(pi) q_s (selected
// parts), the potential at every particle from all the others and their images, so that
// E = 1/2 sum_i q_i phi_i (the self term -beta/sqrt(pi) sum q^2 is the last addend's share).
__global__ void k_unsort(int64_t n, const int *__restrict__ perm, const double *__restrict__ fr,
                         const double *__restrict__ fk, int parts, double *__restrict__ out,
                         const double *__restrict__ pr, const double *__restrict__ pk,
                         const double4_32a *__restrict__ pg, double beta,
                         double *__restrict__ phi_out)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    const bool ur = parts & EWALD_PART_REAL, uk = parts & EWALD_PART_RECIP;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        if (ur) v += fr[3 * s + a];
        if (uk) v += fk[3 * s + a];
        out[3 * i + a] = v;
    }
    if (phi_out) {
        double v = 0.0;
        if (ur) v += pr[s];
        if (uk) v += pk[s];
        if (parts & EWALD_PART_SELF) v += -2.0 * beta / sqrt(kPi) * pg[s].w;
        phi_out[i] = v;
    }
}

// Reciprocal virial tensor from S(k) (the strain derivative of E_recip = sum_{K_half} g |S|^2
// at fixed beta; under a strain eps the volume grows by tr eps and k shrinks by eps k while
// S(k) is unchanged):
//   W_ab = sum_{k in K_half} g(k) |S(k)|^2 [delta_ab - 2 k_a k_b (1/k^2 + 1/(4 beta^2))].
// Block b sums the modes b * 256 + t + j * (gridDim.x * 256) of thread t in order, then a
// fixed tree; part[c * gridDim.x + b] for c = xx, yy, zz, xy, xz, yz.
__global__ void __launch_bounds__(256)
k_recip_virial(int64_t nk, const int *__restrict__ kset, const double *__restrict__ g,
               const double *__restrict__ S, double kf, double c4, double *__restrict__ part)
{
    __shared__ double red[6][256];
    const int t = threadIdx.x;
    double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t u = (int64_t)blockIdx.x * 256 + t; u < nk; u += (int64_t)gridDim.x * 256) {
        const double kx = kf * kset[3 * u], ky = kf * kset[3 * u + 1], kz = kf * kset[3 * u + 2];
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double sr = S[2 * u], si = S[2 * u + 1];
        const double e = g[u] * (sr * sr + si * si);
        const double c = 2.0 * e * (1.0 / k2 + c4);
        w[0] += e - c * kx * kx;
        w[1] += e - c * ky * ky;
        w[2] += e - c * kz * kz;
        w[3] -= c * kx * ky;
        w[4] -= c * kx * kz;
        w[5] -= c * ky * kz;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) red[c][t] = w[c];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) {
#pragma unroll
            for (int c = 0; c < 6; ++c) red[c][t] += red[c][t + o];
        }
        __syncthreads();
    }
    if (t < 6) part[t * gridDim.x + blockIdx.x] = red[t][0];
}

// Virial tensors (one block, fixed order): vir[0..8] real, vir[9..17] reciprocal,
// vir[18..26] self (zero: the self energy does not depend on the positions or the box at
// fixed beta), vir[27..35] their sum; each 3 x 3 row-major and symmetric.
// With Lennard-Jones pairs (lj), their virial (rows 6-11 of vir_tile) is part of the sum
// only.
__global__ void k_virial(int ntile, const double *__restrict__ vir_tile, int64_t vcap,
                         int nblk, const double *__restrict__ vir_part, int parts, int lj,
                         double *__restrict__ vir)
{
    __shared__ double red[256];
    double wr[6], wk[6], wl[6];
    for (int c = 0; c < 6; ++c) {
        wr[c] = (parts & EWALD_PART_REAL) ? block_sum_fixed(vir_tile + c * vcap, ntile, red) : 0.0;
        wk[c] = (parts & EWALD_PART_RECIP) ? block_sum_fixed(vir_part + c * nblk, nblk, red) : 0.0;
        wl[c] = lj ? block_sum_fixed(vir_tile + (6 + c) * vcap, ntile, red) : 0.0;
    }
    if (threadIdx.x == 0) {
        const int ix[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};   // (a, b) -> xx yy zz xy xz yz
        for (int u = 0; u < 9; ++u) {
            vir[u] = wr[ix[u]];
            vir[9 + u] = wk[ix[u]];
            vir[18 + u] = 0.0;
            vir[27 + u] = (wr[ix[u]] + wk[ix[u]]) + wl[ix[u]];
        }
    }
}

__global__ void k_zero_energy(double *e)
{
    if (threadIdx.x < 4) e[threadIdx.x] = 0.0;
}

__global__ void k_zero(double *x, int m)
{
    for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = 0.0;
}

int status_from_bits(int bits)
{
    if (bits & kStNonFinite) return EWALD_E_NONFINITE;
    if (bits & kStTimeout) return EWALD_E_TIMEOUT;
    if (bits & kStNonNeutral) return EWALD_E_NONNEUTRAL;
    if (bits & kStBadType) return EWALD_E_INVAL;
    if (bits & kStRange) return EWALD_E_UNSUPPORTED;
    return EWALD_OK;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return EWALD_OK;
    if (e == cudaErrorMemoryAllocation) return EWALD_E_NOMEM;
    return EWALD_E_CUDA;
}

bool uses_tc(int precision)
{
    return precision == EWALD_MIXED || precision == EWALD_MIXED_BF16;
}

// Drop the captured evaluation graph: its kernels hold pointers to the workspaces and the
// plan's parameters, so it goes whenever either changes.
void graph_reset(Plan &p)
{
    if (p.gexec) {
        if (p.graph_stream) cudaStreamSynchronize(p.graph_stream);
        cudaGraphExecDestroy(p.gexec);
        p.gexec = nullptr;
    }
    p.gkey = Plan::EvalKey();
    p.last_key = Plan::EvalKey();
}

void free_workspace(Plan &p)
{
    graph_reset(p);
    Workspace &ws = p.ws;
    void *ptrs[] = {ws.key, ws.perm, ws.key_sorted, ws.hist, ws.cell_start, ws.cell_total,
                    ws.row_start, ws.perm1, ws.key1, ws.unordered,
                    ws.tiles, ws.tile_off, ws.pg, ws.pl64, ws.pl32, ws.pu,
                    ws.f_real, ws.f_recip, ws.e_tile, ws.qpart, ws.phi_real, ws.phi_recip,
                    ws.vir_tile, ws.vir_part, ws.type_sorted, ws.elj_tile};
    for (void *q : ptrs) pool_free(q, p.side_stream);
    free_recip_simt(p);
    if (uses_tc(p.precision)) free_recip_tc(p);
    int64_t keep_host = ws.cap_host;
    double *hp = ws.h_pos, *hq = ws.h_q, *hf = ws.h_f, *he = ws.h_e;
    ws = Workspace();
    ws.cap_host = keep_host;
    ws.h_pos = hp; ws.h_q = hq; ws.h_f = hf; ws.h_e = he;
}

int binning_chunks(int64_t n, int64_t nrows)
{
    // chunks of 2048 particles (one warp places a chunk in input order), as many as keep the
    // per-chunk histograms over the rows of cells within 2^24 counters, and at most 16384
    // particles a chunk (the scatter keeps a chunk's keys in shared memory)
    int64_t nb = (n + 2047) / 2048;
    const int64_t cap = (int64_t)(1 << 24) / (nrows > 0 ? nrows : 1);
    if (nb > cap) nb = cap > 0 ? cap : 1;
    if ((n + nb - 1) / nb > 16384) nb = (n + 16383) / 16384;
    return nb < 1 ? 1 : (int)nb;
}

}  // namespace

// Library-owned stream-ordered memory pool of the current device.  Plans allocate their
// workspaces from it, so a freed workspace is kept for the next plan instead of going back
// to the driver (the serving loop creates and drops plans per request).
cudaMemPool_t lib_pool()
{
    static cudaMemPool_t pools[64] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pl = nullptr;
        if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) return nullptr;
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pl;
    }
    return pools[dev];
}

// Opt a kernel into the largest dynamic shared memory a block may have on the current
// device, once per (kernel, device).  The attribute belongs to the kernel, not to a plan or a
// thread, so it is never set to a launch's own size: the server launches several plans from
// several threads, and a smaller value set by one of them between another's setting and its
// launch would fail that launch.
cudaError_t smem_optin(const void *func, size_t *max_dynamic)
{
    struct Done { const void *f; int dev; int bytes; };
    static std::mutex mu;
    static std::vector<Done> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    for (const Done &d : done)
        if (d.f == func && d.dev == dev) {
            if (max_dynamic) *max_dynamic = (size_t)d.bytes;
            return cudaSuccess;
        }
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
    const int bytes = optin - (int)fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return e;
    done.push_back(Done{func, dev, bytes});
    if (max_dynamic) *max_dynamic = (size_t)bytes;
    return cudaSuccess;
}

cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st)
{
    cudaMemPool_t pl = lib_pool();
    if (!pl) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(ptr, bytes < 256 ? 256 : bytes, pl, st);
}

void pool_free(void *ptr, cudaStream_t st)
{
    if (ptr) cudaFreeAsync(ptr, st);
}

namespace {

template <class P>
cudaError_t dmalloc(Plan &pl, P **p, size_t bytes)
{
    return pool_alloc((void **)p, bytes, pl.side_stream);
}

cudaError_t grow_workspace(Plan &p, int64_t n)
{
    // The cell grid follows the density of this evaluation's particle count (not the
    // capacity of the workspace), so that a system's results do not depend on what the plan
    // evaluated before; buffers sized by the particle count keep the larger capacity.
    int nc = 1, w = 0;
    cell_grid(p.L, p.rc, n, nc, w);
    if (n <= p.ws.cap_n && nc == p.nc && w == p.w) return cudaSuccess;
    if (n <= p.ws.cap_n) {
        // another grid in the same buffers where they are large enough
        const int64_t cells = (int64_t)nc * nc * nc, rows = (int64_t)nc * nc;
        const int nb = binning_chunks(p.ws.cap_n, rows);
        const int nc0 = p.nc, w0 = p.w;
        p.nc = nc;
        p.w = w;
        const int64_t tiles = real_tile_capacity(p, p.ws.cap_n);
        p.nc = nc0;
        p.w = w0;
        if (cells <= p.ws.cap_cells && rows <= p.ws.cap_rows && tiles <= p.ws.cap_tiles &&
            (int64_t)nb * rows <= p.ws.cap_hist) {
            cudaError_t e = cudaStreamSynchronize(p.last_stream ? p.last_stream : 0);
            if (e != cudaSuccess) return e;
            if ((e = cudaStreamSynchronize(p.side_stream)) != cudaSuccess) return e;
            graph_reset(p);
            p.nc = nc;
            p.w = w;
            p.ncells = (int)cells;
            p.cell_side = p.L / nc;
            p.ws.nb = nb;
            return cudaSuccess;
        }
    }
    const int64_t cap = n > p.ws.cap_n ? n : p.ws.cap_n;
    cudaError_t e = cudaStreamSynchronize(p.last_stream ? p.last_stream : 0);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(p.side_stream)) != cudaSuccess) return e;
    free_workspace(p);
    p.nc = nc;
    p.w = w;
    p.ncells = p.nc * p.nc * p.nc;
    p.cell_side = p.L / p.nc;
    p.real_tile = real_tile_for(p.w, (double)n / p.ncells);
    Workspace &ws = p.ws;
    const int nb = binning_chunks(cap, (int64_t)p.nc * p.nc);
    const int64_t tiles = real_tile_capacity(p, cap);
    const int64_t qblocks = (cap + 255) / 256;
#define EW_TRY(x) do { if ((e = (x)) != cudaSuccess) { free_workspace(p); return e; } } while (0)
    EW_TRY(dmalloc(p, &ws.key, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.perm, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.key_sorted, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.hist, sizeof(int) * (size_t)nb * p.nc * p.nc));
    EW_TRY(dmalloc(p, &ws.cell_start, sizeof(int) * (p.ncells + 1)));
    EW_TRY(dmalloc(p, &ws.cell_total, sizeof(int) * p.nc * p.nc));
    EW_TRY(dmalloc(p, &ws.row_start, sizeof(int) * (p.nc * p.nc + 1)));
    EW_TRY(dmalloc(p, &ws.perm1, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.key1, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.tiles, sizeof(int2) * tiles));
    EW_TRY(dmalloc(p, &ws.tile_off, sizeof(int) * (p.nc * p.nc + 1)));
    EW_TRY(dmalloc(p, &ws.unordered, sizeof(int)));
    EW_TRY(dmalloc(p, &ws.pg, sizeof(double4_32a) * cap));
    if (p.precision == EWALD_FP64) EW_TRY(dmalloc(p, &ws.pl64, sizeof(double4_32a) * cap));
    else EW_TRY(dmalloc(p, &ws.pl32, sizeof(float4) * cap));
    EW_TRY(dmalloc(p, &ws.pu, sizeof(uint4) * cap));
    EW_TRY(dmalloc(p, &ws.f_real, sizeof(double) * 3 * cap));
    EW_TRY(dmalloc(p, &ws.phi_real, sizeof(double) * cap));
    EW_TRY(dmalloc(p, &ws.phi_recip, sizeof(double) * cap));
    EW_TRY(dmalloc(p, &ws.f_recip, sizeof(double) * 3 * cap));
    EW_TRY(dmalloc(p, &ws.e_tile, sizeof(double) * tiles));
    EW_TRY(dmalloc(p, &ws.vir_tile, sizeof(double) * 12 * tiles));
    EW_TRY(dmalloc(p, &ws.elj_tile, sizeof(double) * tiles));
    EW_TRY(dmalloc(p, &ws.type_sorted, sizeof(int) * cap));
    EW_TRY(dmalloc(p, &ws.vir_part, sizeof(double) * 6 * kVirBlocks));
    EW_TRY(dmalloc(p, &ws.qpart, sizeof(double) * 3 * qblocks));
    ws.cap_n = cap;
    ws.nb = nb;
    ws.cap_cells = p.ncells;
    ws.cap_rows = (int64_t)p.nc * p.nc;
    ws.cap_tiles = tiles;
    ws.cap_hist = (int64_t)nb * p.nc * p.nc;
    if (uses_tc(p.precision)) EW_TRY(alloc_recip_tc(p, cap));
    else EW_TRY(alloc_recip_simt(p, cap));
#undef EW_TRY
    // allocations are ordered on the side stream; make them visible to every stream
    return cudaStreamSynchronize(p.side_stream);
}

cudaError_t pipeline(Plan &p, int64_t n, const double *pos, const double *q, double *forces,
                     double *energy_dev, int parts, cudaStream_t st, bool clear_status = true,
                     double *phi = nullptr, double *vir = nullptr)
{
    cudaError_t e;
    Workspace &ws = p.ws;
    p.launches = 0;
    // a failed call of an earlier evaluation (e.g. a rejected launch configuration) must not be
    // reported against this one
    (void)cudaGetLastError();
    prof_mark(p, kEvStart, st);
    p.prof_bs = false;
    if (clear_status && (e = cudaMemsetAsync(p.d_status, 0, sizeof(int), st)) != cudaSuccess)
        return e;
    if ((e = launch_binning(p, n, pos, q, st)) != cudaSuccess) return e;
    const bool lj = p.lj_ntypes > 0 && (parts & EWALD_PART_REAL);
    if (lj) {
        k_gather_type<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ws.perm, p.lj_type,
                                                                   p.lj_ntypes, ws.type_sorted,
                                                                   p.d_status);
        p.launches += 1;
    }
    prof_mark(p, kEvBinned, st);
    const int64_t tiles = real_tile_capacity(p, n);
    if ((e = cudaMemsetAsync(ws.e_tile, 0, sizeof(double) * tiles, st)) != cudaSuccess) return e;
    if (vir && (e = cudaMemsetAsync(ws.vir_tile, 0, sizeof(double) * (lj ? 12 : 6) * tiles, st)) != cudaSuccess)
        return e;
    if (lj && (e = cudaMemsetAsync(ws.elj_tile, 0, sizeof(double) * tiles, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(p.e_recip_part, 0, sizeof(double) * p.e_recip_count, st)) != cudaSuccess) return e;
    const bool do_recip = parts & EWALD_PART_RECIP;
    const bool spme = p.spme != nullptr;
    if (do_recip && !spme && uses_tc(p.precision) &&
        (e = launch_recip_tc_operands(p, n, st)) != cudaSuccess)
        return e;
    if (do_recip) {
        if ((e = cudaEventRecord(p.ev_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(p.side_stream, p.ev_fork, 0)) != cudaSuccess) return e;
        e = spme ? launch_recip_spme(p, n, p.side_stream)
                 : uses_tc(p.precision) ? launch_recip_tc(p, n, p.side_stream)
                                        : launch_recip_simt(p, n, p.side_stream);
        if (e != cudaSuccess) return e;
        if (vir && !spme) {   // (the SPME spectrum pass writes its own virial partials)
            k_recip_virial<<<kVirBlocks, 256, 0, p.side_stream>>>(
                p.nk, p.kset_d, p.g_d, p.S_d, 2.0 * kPi / p.L, 0.25 / (p.beta * p.beta),
                ws.vir_part);
            p.launches += 1;
        }
        if ((e = cudaEventRecord(p.ev_join, p.side_stream)) != cudaSuccess) return e;
    }
    prof_mark(p, kEvRealStart, st);
    if (parts & EWALD_PART_REAL) {
        if ((e = launch_real(p, n, st, vir != nullptr)) != cudaSuccess) return e;
    }
    prof_mark(p, kEvRealEnd, st);
    if (do_recip) {
        if ((e = cudaStreamWaitEvent(st, p.ev_join, 0)) != cudaSuccess) return e;
    }
    prof_mark(p, kEvJoined, st);
    int erc = p.e_recip_count;
    const double *erp = p.e_recip_part;
    if (spme) erp = spme_energy_parts(p, &erc);
    k_energy<<<1, 256, 0, st>>>((int)tiles, ws.e_tile, (int)((n + 255) / 256), ws.qpart,
                                erc, erp, p.beta, parts,
                                lj ? ws.elj_tile : nullptr, (spme && do_recip) ? 1 : 0,
                                energy_dev, p.d_status);
    k_unsort<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ws.perm, ws.f_real, ws.f_recip,
                                                          parts, forces, ws.phi_real,
                                                          ws.phi_recip, ws.pg, p.beta, phi);
    p.launches += 2;
    if (vir) {
        int vrc = kVirBlocks;
        const double *vrp = ws.vir_part;
        if (spme) vrp = spme_virial_parts(p, &vrc);
        k_virial<<<1, 256, 0, st>>>((int)tiles, ws.vir_tile, tiles, vrc, vrp, parts, lj ? 1 : 0,
                                    vir);
        p.launches += 1;
    }
    prof_mark(p, kEvFinal, st);
    p.prof_valid = p.prof;
    p.prof_recip = p.prof && do_recip;
    p.last_stream = st;
    return cudaGetLastError();
}

}  // namespace

// One evaluation.  An evaluation with the same arguments (sizes and buffers) as the one
// before it is captured once into a CUDA graph, on the plan's graph stream, and replayed from
// then on: the ~20 launches of the pipeline (two streams) become one graph launch.  A first
// call, a call with new buffers, a call while profiling, and a call on a stream that is
// itself being captured run the pipeline directly.
cudaError_t evaluate(Plan &p, int64_t n, const double *pos, const double *q, double *forces,
                     double *energy_dev, int parts, cudaStream_t st, bool clear_status,
                     double *phi, double *vir)
{
    cudaError_t e = grow_workspace(p, n);
    if (e != cudaSuccess) return e;
    Plan::EvalKey key;
    key.n = n; key.pos = pos; key.q = q; key.forces = forces; key.energy = energy_dev;
    key.parts = parts; key.clear = clear_status; key.phi = phi; key.vir = vir;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return e;
    const bool repeat = key == p.last_key;
    p.last_key = key;
    // (SPME evaluations run directly: their transforms are library calls)
    if (p.prof || !p.graph_stream || cap != cudaStreamCaptureStatusNone || !repeat || p.spme)
        return pipeline(p, n, pos, q, forces, energy_dev, parts, st, clear_status, phi, vir);
    if ((e = cudaEventRecord(p.ev_gin, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(p.graph_stream, p.ev_gin, 0)) != cudaSuccess) return e;
    if (!(p.gexec && key == p.gkey)) {
        // capture the pipeline on the graph stream
        (void)cudaGetLastError();
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(p.graph_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return e;
        cudaError_t ep = pipeline(p, n, pos, q, forces, energy_dev, parts, p.graph_stream,
                                  clear_status, phi, vir);
        cudaError_t ec = cudaStreamEndCapture(p.graph_stream, &g);
        if (ep != cudaSuccess || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            (void)cudaGetLastError();
            p.gkey = Plan::EvalKey();
            return ep != cudaSuccess ? ep : (ec != cudaSuccess ? ec : cudaErrorUnknown);
        }
        const int launches = p.launches;
        bool ok = false;
        if (p.gexec) {
            cudaGraphExecUpdateResultInfo info;
            ok = cudaGraphExecUpdate(p.gexec, g, &info) == cudaSuccess;
            if (!ok) {
                (void)cudaGetLastError();
                cudaGraphExecDestroy(p.gexec);
                p.gexec = nullptr;
            }
        }
        if (!ok) e = cudaGraphInstantiate(&p.gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p.gexec = nullptr; p.gkey = Plan::EvalKey(); return e; }
        p.gkey = key;
        p.g_launches = launches;
    }
    if ((e = cudaGraphLaunch(p.gexec, p.graph_stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(p.ev_gout, p.graph_stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(st, p.ev_gout, 0)) != cudaSuccess) return e;
    p.launches = p.g_launches;
    p.prof_valid = false;
    p.last_stream = st;
    return cudaSuccess;
}

size_t plan_footprint(const Plan &p, int64_t n)
{
    int nc = 1, w = 0;
    cell_grid(p.L, p.rc, n, nc, w);
    const int nb = binning_chunks(n, (int64_t)nc * nc);
    const size_t ncells = (size_t)nc * nc * nc;
    const int64_t ts = w == 0 ? 32 : 32 / real_tile_for(w, (double)n / ncells);
    const int64_t tiles = w == 0 ? (n + 31) / 32 : n / ts + (int64_t)nc * nc + 1;
    size_t b = 0;
    const size_t nrows = (size_t)nc * nc;
    b += sizeof(int) * 5 * (size_t)n + sizeof(int) * (size_t)nb * nrows;
    b += sizeof(int) * (ncells + 1 + 2 * nrows + 1) + sizeof(int2) * tiles + sizeof(int) * (nrows + 1);
    b += (sizeof(double4_32a) + (p.precision == EWALD_FP64 ? sizeof(double4_32a) : sizeof(float4)) + sizeof(uint4)) * (size_t)n;
    b += sizeof(double) * 8 * (size_t)n + sizeof(double) * 14 * tiles + sizeof(double) * 3 * ((n + 255) / 256);
    b += sizeof(int) * (size_t)n + sizeof(int);
    b += sizeof(double) * 6 * kVirBlocks;
    b += uses_tc(p.precision) ? recip_tc_bytes(p, n) : recip_simt_bytes(p, n);
    b += sizeof(double) * 3 * (size_t)p.nk + sizeof(int) * 3 * (size_t)p.nk + sizeof(RowInfo) * p.R;
    b += sizeof(double) * 32 * (size_t)p.R;
    return b;
}

}  // namespace ew

// ---- plan construction ------------------------------------------------------------------

static void build_rows(Plan &p)
{
    // Rows (m_y, m_z) of the half plane; koff is each row's offset in the K_half order
    // (m_z, then m_y, then m_x ascending).  The rows are then processed in order of
    // decreasing m_y^2 + m_z^2: the coefficients g(k) |S(k)| grow along that order, so the
    // back-scatter sums over rows add the small terms before the large ones.
    const int k = p.kmax;
    p.rows_h.clear();
    int64_t koff = 0;
    for (int mz = 0; mz <= k; ++mz)
        for (int my = -k; my <= k; ++my) {
            if (my * my + mz * mz > k * k) continue;
            if (mz == 0 && my < 0) continue;
            int rem = k * k - my * my - mz * mz;
            int nx = (int)floor(sqrt((double)rem));
            while ((nx + 1) * (nx + 1) <= rem) ++nx;
            while (nx * nx > rem) --nx;
            RowInfo r;
            r.my = my; r.mz = mz; r.nxmax = nx; r.koff = (int)koff;
            koff += (my == 0 && mz == 0) ? nx : 2 * nx + 1;
            p.rows_h.push_back(r);
        }
    std::stable_sort(p.rows_h.begin(), p.rows_h.end(), [](const RowInfo &a, const RowInfo &b) {
        return a.my * a.my + a.mz * a.mz > b.my * b.my + b.mz * b.mz;
    });
    p.R = (int)p.rows_h.size();
    p.nk = koff;
}

// Cell grid of the real-space pairs: nc^3 cubes of side L / nc, a stencil of |dy|, |dz| <= w
// rows with w = ceil(r_c nc / L), and 2 w + 1 <= nc so that the stencil's rows (and the
// cells of a row a target can reach) are distinct.  The side aims at max(1.33 rho^-1/3,
// r_c / 5): about 2.4 particles per cell or more, and at most ~11 rows across the cutoff
// disk, so that each target's candidate ranges follow its cutoff sphere closely (the pair
// kernel takes the cells of every row within each target's own reach) while a row holds
// enough candidates to pay for its set-up (measured on GB300, 32,768 ions at r_c = 4: cells
// of side 1, 1.33, 1.6, 2 take 0.172, 0.129, 0.135, 0.125 ms; at long cutoffs, sides r_c / 6,
// r_c / 7, r_c / 8 test fewer candidates per partner but walk up to twice the rows, and were no
// faster at 262,144 and 2,097,152 ions).  Without the density (plan set-up)
// the side is r_c / 2; the grid is chosen again once the particle count is known.  Boxes too
// small for such a stencil use the all-pairs mode (w = 0, one cell).
static void cell_grid(double L, double rc, int64_t n, int &nc_out, int &w_out)
{
    const double rho = n > 0 ? (double)n / (L * L * L) : 0.0;
    double s_t = rho > 0 ? fmax(1.33 * pow(rho, -1.0 / 3.0), rc / 5.0) : rc / 2.0;
    int nc = (int)floor(L / s_t);
    if (nc > kMaxCellsPerSide) nc = kMaxCellsPerSide;   // a row's counts in shared memory
    w_out = 0;
    nc_out = 1;
    for (; nc >= 3; --nc) {
        const int w = (int)ceil(rc * nc / L * (1.0 - 1e-12));
        if (w >= 1 && 2 * w + 1 <= nc) {
            nc_out = nc;
            w_out = w;
            return;
        }
    }
}

static void choose_cells(Plan &p)
{
    cell_grid(p.L, p.rc, 0, p.nc, p.w);
    p.ncells = p.nc * p.nc * p.nc;
    p.cell_side = p.L / p.nc;
}

namespace ew {

int plan_setup_host(Plan &p, double L, double beta, double rc, int kmax, int precision)
{
    if (!(L > 0) || !isfinite(L) || !(beta > 0) || !isfinite(beta)) return EWALD_E_INVAL;
    if (!(rc > 0) || !(rc <= 0.5 * L)) return EWALD_E_CUTOFF;
    if (kmax < 1) return EWALD_E_INVAL;
    if (kmax > 127) return EWALD_E_UNSUPPORTED;
    if (precision < EWALD_FP64 || precision > EWALD_FP32) return EWALD_E_INVAL;
    p.L = L; p.beta = beta; p.rc = rc; p.kmax = kmax; p.precision = precision;
    choose_cells(p);
    build_rows(p);
    p.e_recip_count = uses_tc(precision) ? recip_tc_energy_parts(p) : p.R;
    return EWALD_OK;
}

// The modes of every row in K_half order (m_x ascending; m_x > 0 only on the row (0, 0)) and
// g(k) = 4 pi exp(-k^2 / (4 beta^2)) / (V k^2) (C_k of Eq. 3), k = 2 pi m / L.  One block per
// row.
__global__ void k_plan_tables(const RowInfo *__restrict__ rows, double tpl, double V,
                              double beta, int *__restrict__ kset, double *__restrict__ g)
{
    const RowInfo r = rows[blockIdx.x];
    const int lo = (r.my == 0 && r.mz == 0) ? 1 : -r.nxmax;
    const int cnt = r.nxmax - lo + 1;
    const double inv4b2 = 1.0 / (4.0 * beta * beta);
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const int mx = lo + t;
        const int64_t idx = (int64_t)r.koff + t;
        kset[3 * idx + 0] = mx;
        kset[3 * idx + 1] = r.my;
        kset[3 * idx + 2] = r.mz;
        const double m2 = (double)mx * mx + (double)r.my * r.my + (double)r.mz * r.mz;
        const double k2 = tpl * tpl * m2;
        g[idx] = 4.0 * kPi * exp(-k2 * inv4b2) / (V * k2);
    }
}

// Upload the row table and k list of the current parameters, (re)allocating the plan-level
// arrays when they grow.  Runs on the side stream and waits for it.
static cudaError_t plan_upload(Plan &p)
{
    cudaError_t e;
    cudaStream_t st = p.side_stream;
    if (p.R > p.cap_R) {
        pool_free(p.rows_d, st); pool_free(p.e_recip_part, st); pool_free(p.fperm_d, st);
        p.rows_d = nullptr; p.e_recip_part = nullptr; p.fperm_d = nullptr; p.cap_R = 0;
        if ((e = pool_alloc((void **)&p.rows_d, sizeof(RowInfo) * p.R, st)) != cudaSuccess) return e;
        if ((e = pool_alloc((void **)&p.fperm_d, sizeof(int) * p.R, st)) != cudaSuccess) return e;
        // room for the partial reciprocal energies of either path (at most 32 per row)
        if ((e = pool_alloc((void **)&p.e_recip_part, sizeof(double) * 32 * (size_t)p.R, st)) != cudaSuccess) return e;
        p.cap_R = p.R;
    }
    if (p.nk > p.cap_nk) {
        pool_free(p.kset_d, st); pool_free(p.S_d, st); pool_free(p.g_d, st);
        p.kset_d = nullptr; p.S_d = nullptr; p.g_d = nullptr; p.cap_nk = 0;
        if ((e = pool_alloc((void **)&p.kset_d, sizeof(int) * 3 * p.nk, st)) != cudaSuccess) return e;
        if ((e = pool_alloc((void **)&p.S_d, sizeof(double) * 2 * p.nk, st)) != cudaSuccess) return e;
        if ((e = pool_alloc((void **)&p.g_d, sizeof(double) * p.nk, st)) != cudaSuccess) return e;
        p.cap_nk = p.nk;
    }
    if ((e = cudaMemcpyAsync(p.rows_d, p.rows_h.data(), sizeof(RowInfo) * p.R, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    // forward order of the rows: decreasing n_x,max (the reverse of the row order), so that
    // each 64-row tile of the forward product needs only the m_x columns of its first row
    std::vector<int> fperm(p.R);
    for (int i = 0; i < p.R; ++i) fperm[i] = p.R - 1 - i;
    if ((e = cudaMemcpyAsync(p.fperm_d, fperm.data(), sizeof(int) * p.R, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    // the k list and g(k) of every mode, generated on the device from the row table
    k_plan_tables<<<p.R, 128, 0, st>>>(p.rows_d, 2.0 * kPi / p.L, p.L * p.L * p.L, p.beta,
                                       p.kset_d, p.g_d);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.S_d, 0, sizeof(double) * 2 * p.nk, st)) != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

int plan_reconfigure(ewald_plan *h, double L, double beta, double rc, int kmax, int precision)
{
    Plan &p = h->p;
    Plan probe;
    probe.num_sms = p.num_sms;
    int s = plan_setup_host(probe, L, beta, rc, kmax, precision);
    if (s != EWALD_OK) return s;
    if (p.last_stream) cudaStreamSynchronize(p.last_stream);
    cudaStreamSynchronize(p.side_stream);
    // the workspace is kept where the k tables keep their shape; its cell grid is checked
    // against the particle count of the next evaluation (grow_workspace)
    const bool same_shape = p.ws.cap_n > 0 && probe.R == p.R && probe.kmax == p.kmax &&
                            probe.precision == p.precision;
    const int nc0 = p.nc, w0 = p.w;
    graph_reset(p);
    if (!same_shape) free_workspace(p);
    plan_setup_host(p, L, beta, rc, kmax, precision);
    if (same_shape) {
        p.nc = nc0;
        p.w = w0;
        p.ncells = nc0 * nc0 * nc0;
        p.cell_side = L / nc0;
    }
    return cuda_status(plan_upload(p));
}

}  // namespace ew

static void destroy_plan(ewald_plan *h)
{
    Plan &p = h->p;
    if (p.last_stream) cudaStreamSynchronize(p.last_stream);
    if (p.side_stream) {
        cudaStreamSynchronize(p.side_stream);
        free_workspace(p);
        pool_free(p.rows_d, p.side_stream); pool_free(p.kset_d, p.side_stream);
        pool_free(p.fperm_d, p.side_stream);
        pool_free(p.S_d, p.side_stream); pool_free(p.e_recip_part, p.side_stream);
        pool_free(p.g_d, p.side_stream);
        pool_free(p.energy_d, p.side_stream); pool_free(p.d_status, p.side_stream);
        pool_free(p.lj_tab_d, p.side_stream);
        pool_free(p.ws.h_pos, p.side_stream); pool_free(p.ws.h_q, p.side_stream);
        pool_free(p.ws.h_f, p.side_stream);
        cudaStreamSynchronize(p.side_stream);
    }
    graph_reset(p);
    spme_free(p);
    if (p.h_status) cudaFreeHost(p.h_status);
    if (p.side_stream) cudaStreamDestroy(p.side_stream);
    if (p.graph_stream) cudaStreamDestroy(p.graph_stream);
    if (p.ev_gin) cudaEventDestroy(p.ev_gin);
    if (p.ev_gout) cudaEventDestroy(p.ev_gout);
    if (p.ev_fork) cudaEventDestroy(p.ev_fork);
    if (p.ev_join) cudaEventDestroy(p.ev_join);
    for (cudaEvent_t ev : p.ev)
        if (ev) cudaEventDestroy(ev);
    delete h;
}

extern "C" int ewald_create(double L, double beta, double r_c, int k_max, int precision,
                            ewald_plan_t *out)
{
    if (!out) return EWALD_E_INVAL;
    *out = nullptr;
    Plan probe;
    int s = plan_setup_host(probe, L, beta, r_c, k_max, precision);
    if (s != EWALD_OK) return s;
    ewald_plan *h = new (std::nothrow) ewald_plan();
    if (!h) return EWALD_E_NOMEM;
    Plan &p = h->p;
    plan_setup_host(p, L, beta, r_c, k_max, precision);
    cudaGetDevice(&p.device);
    cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device);
    if (p.num_sms < 1) p.num_sms = 1;
    cudaError_t e = cudaSuccess;
#define EW_C(x) do { if ((e = (x)) != cudaSuccess) { destroy_plan(h); return cuda_status(e); } } while (0)
    EW_C(cudaStreamCreateWithFlags(&p.side_stream, cudaStreamNonBlocking));
    EW_C(cudaEventCreateWithFlags(&p.ev_fork, cudaEventDisableTiming));
    EW_C(cudaEventCreateWithFlags(&p.ev_join, cudaEventDisableTiming));
    EW_C(cudaStreamCreateWithFlags(&p.graph_stream, cudaStreamNonBlocking));
    EW_C(cudaEventCreateWithFlags(&p.ev_gin, cudaEventDisableTiming));
    EW_C(cudaEventCreateWithFlags(&p.ev_gout, cudaEventDisableTiming));
    EW_C(cudaHostAlloc((void **)&p.h_status, sizeof(int), cudaHostAllocDefault));
    EW_C(pool_alloc((void **)&p.energy_d, sizeof(double) * 4, p.side_stream));
    EW_C(pool_alloc((void **)&p.d_status, sizeof(int), p.side_stream));
    EW_C(cudaMemsetAsync(p.d_status, 0, sizeof(int), p.side_stream));
    EW_C(plan_upload(p));
#undef EW_C
    *out = h;
    return EWALD_OK;
}

extern "C" void ewald_destroy(ewald_plan_t plan)
{
    if (plan) destroy_plan(plan);
}

static int validate_call(ewald_plan_t plan, int64_t n, const void *pos, const void *q,
                         const void *forces)
{
    if (!plan) return EWALD_E_INVAL;
    if (n < 0 || n > (int64_t)INT32_MAX / 4) return EWALD_E_INVAL;
    if (n > 0 && (!pos || !q || !forces)) return EWALD_E_INVAL;
    return EWALD_OK;
}

extern "C" int ewald_compute_async(ewald_plan_t plan, int64_t n, const double *pos,
                                   const double *q, double *forces, double *energy_dev,
                                   int parts, void *stream)
{
    int s = validate_call(plan, n, pos, q, forces);
    if (s != EWALD_OK) return s;
    if (!energy_dev || (parts & ~EWALD_PART_ALL)) return EWALD_E_INVAL;
    Plan &p = plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        k_zero_energy<<<1, 32, 0, st>>>(energy_dev);
        p.last_stream = st;
        return cuda_status(cudaGetLastError());
    }
    cudaError_t e = evaluate(p, n, pos, q, forces, energy_dev, parts, st, true);
    return cuda_status(e);
}

extern "C" int ewald_compute_phi_async(ewald_plan_t plan, int64_t n, const double *pos,
                                       const double *q, double *forces, double *phi_dev,
                                       double *energy_dev, int parts, void *stream)
{
    int s = validate_call(plan, n, pos, q, forces);
    if (s != EWALD_OK) return s;
    if (!energy_dev || (parts & ~EWALD_PART_ALL) || (n > 0 && !phi_dev)) return EWALD_E_INVAL;
    Plan &p = plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        k_zero_energy<<<1, 32, 0, st>>>(energy_dev);
        p.last_stream = st;
        return cuda_status(cudaGetLastError());
    }
    return cuda_status(evaluate(p, n, pos, q, forces, energy_dev, parts, st, true, phi_dev));
}

extern "C" int ewald_compute_virial_async(ewald_plan_t plan, int64_t n, const double *pos,
                                          const double *q, double *forces, double *virial_dev,
                                          double *energy_dev, int parts, void *stream)
{
    int s = validate_call(plan, n, pos, q, forces);
    if (s != EWALD_OK) return s;
    if (!energy_dev || !virial_dev || (parts & ~EWALD_PART_ALL)) return EWALD_E_INVAL;
    Plan &p = plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        k_zero_energy<<<1, 32, 0, st>>>(energy_dev);
        k_zero<<<1, 64, 0, st>>>(virial_dev, 36);
        p.last_stream = st;
        return cuda_status(cudaGetLastError());
    }
    return cuda_status(evaluate(p, n, pos, q, forces, energy_dev, parts, st, true, nullptr,
                                virial_dev));
}

extern "C" int ewald_set_lj(ewald_plan_t plan, int ntypes, const double *epsilon,
                            const double *sigma, const int32_t *type_dev)
{
    if (!plan || ntypes < 0 || ntypes > EWALD_LJ_MAX_TYPES) return EWALD_E_INVAL;
    Plan &p = plan->p;
    if (ntypes == 0) {
        if (p.last_stream) cudaStreamSynchronize(p.last_stream);
        graph_reset(p);
        p.lj_ntypes = 0;
        p.lj_type = nullptr;
        return EWALD_OK;
    }
    if (!epsilon || !sigma || !type_dev) return EWALD_E_INVAL;
    double tab[EWALD_LJ_MAX_TYPES * EWALD_LJ_MAX_TYPES * 4];
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b) {
            const double e = epsilon[a * ntypes + b], s = sigma[a * ntypes + b];
            if (!(e >= 0) || !isfinite(e) || !(s > 0) || !isfinite(s)) return EWALD_E_INVAL;
            if (e != epsilon[b * ntypes + a] || s != sigma[b * ntypes + a]) return EWALD_E_INVAL;
            double *t = tab + 4 * (a * ntypes + b);
            t[0] = s * s;
            t[1] = 4.0 * e;
            t[2] = 24.0 * e;
            t[3] = 0.0;
        }
    // the graph of the last evaluation and a running evaluation may still read the old table
    if (p.last_stream) cudaStreamSynchronize(p.last_stream);
    cudaStreamSynchronize(p.side_stream);
    graph_reset(p);
    cudaError_t e = cudaSuccess;
    if (!p.lj_tab_d) {
        e = pool_alloc((void **)&p.lj_tab_d, sizeof(tab), p.side_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p.side_stream);
        if (e != cudaSuccess) { p.lj_tab_d = nullptr; return cuda_status(e); }
    }
    e = cudaMemcpy(p.lj_tab_d, tab, sizeof(double) * 4 * ntypes * ntypes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
    p.lj_ntypes = ntypes;
    p.lj_type = reinterpret_cast<const int *>(type_dev);
    return EWALD_OK;
}

extern "C" int ewald_set_near_pairs(ewald_plan_t plan, int double_float)
{
    if (!plan || (double_float != 0 && double_float != 1)) return EWALD_E_INVAL;
    Plan &p = plan->p;
    if (p.last_stream) cudaStreamSynchronize(p.last_stream);
    if (p.side_stream) cudaStreamSynchronize(p.side_stream);
    // the captured graph holds the kernel of the old mode
    graph_reset(p);
    p.near_df = double_float == 1;
    return EWALD_OK;
}

extern "C" int ewald_set_spme(ewald_plan_t plan, int K, int order)
{
    if (!plan || K < 0) return EWALD_E_INVAL;
    Plan &p = plan->p;
    if (p.last_stream) cudaStreamSynchronize(p.last_stream);
    if (p.side_stream) cudaStreamSynchronize(p.side_stream);
    graph_reset(p);
    return spme_set(p, K, order);
}

extern "C" int ewald_probe_timeout(ewald_plan_t plan, void *stream)
{
    if (!plan) return EWALD_E_INVAL;
    return cuda_status(launch_wait_probe(plan->p, (cudaStream_t)stream));
}

extern "C" int ewald_status_sync(ewald_plan_t plan)
{
    if (!plan) return EWALD_E_INVAL;
    Plan &p = plan->p;
    cudaError_t e = cudaStreamSynchronize(p.last_stream);
    if (e != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpy(p.h_status, p.d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_status(e);
    int bits = *p.h_status;
    cudaMemset(p.d_status, 0, sizeof(int));
    return status_from_bits(bits);
}

extern "C" int ewald_compute(ewald_plan_t plan, int64_t n, const double *pos, const double *q,
                             double *forces, double energy[4], void *stream)
{
    if (!energy) return EWALD_E_INVAL;
    int s = ewald_compute_async(plan, n, pos, q, forces, plan ? plan->p.energy_d : nullptr,
                                EWALD_PART_ALL, stream);
    if (s != EWALD_OK) return s;
    Plan &p = plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(energy, p.energy_d, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemcpyAsync(p.h_status, p.d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_status(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e);
    return status_from_bits(n > 0 ? *p.h_status : 0);
}

extern "C" int ewald_compute_host(ewald_plan_t plan, int64_t n, const double *pos_host,
                                  const double *q_host, double *forces_host,
                                  double energy_host[4], void *stream)
{
    int s = validate_call(plan, n, pos_host, q_host, forces_host);
    if (s != EWALD_OK || !energy_host) return s != EWALD_OK ? s : EWALD_E_INVAL;
    Plan &p = plan->p;
    Workspace &ws = p.ws;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (n > ws.cap_host) {
        if (p.last_stream) cudaStreamSynchronize(p.last_stream);
        cudaStreamSynchronize(p.side_stream);
        pool_free(ws.h_pos, p.side_stream); pool_free(ws.h_q, p.side_stream);
        pool_free(ws.h_f, p.side_stream);
        ws.h_pos = ws.h_q = ws.h_f = nullptr;
        ws.cap_host = 0;
        if ((e = pool_alloc((void **)&ws.h_pos, sizeof(double) * 3 * n, p.side_stream)) != cudaSuccess) return cuda_status(e);
        if ((e = pool_alloc((void **)&ws.h_q, sizeof(double) * n, p.side_stream)) != cudaSuccess) return cuda_status(e);
        if ((e = pool_alloc((void **)&ws.h_f, sizeof(double) * 3 * n, p.side_stream)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaStreamSynchronize(p.side_stream)) != cudaSuccess) return cuda_status(e);
        ws.cap_host = n;
    }
    if (n > 0) {
        if ((e = cudaMemcpyAsync(ws.h_pos, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_status(e);
        if ((e = cudaMemcpyAsync(ws.h_q, q_host, sizeof(double) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_status(e);
    }
    s = ewald_compute(plan, n, ws.h_pos, ws.h_q, ws.h_f, energy_host, stream);
    if (s != EWALD_OK) return s;
    if (n > 0) {
        if ((e = cudaMemcpyAsync(forces_host, ws.h_f, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_status(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e);
    }
    return EWALD_OK;
}

extern "C" int ewald_profile(ewald_plan_t plan, int enable, double times_ms[EWALD_PROFILE_TIMES],
                             int *launches)
{
    if (!plan) return EWALD_E_INVAL;
    Plan &p = plan->p;
    if (enable == 1 && !p.ev[0]) {
        for (cudaEvent_t &ev : p.ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    if (enable >= 0) {
        p.prof = enable == 1;
        if (!p.prof) p.prof_valid = false;
    }
    if (launches) *launches = p.launches;
    if (times_ms) {
        for (int i = 0; i < EWALD_PROFILE_TIMES; ++i) times_ms[i] = 0.0;
        if (!p.prof_valid) return EWALD_OK;
        cudaError_t e = cudaEventSynchronize(p.ev[kEvFinal]);
        if (e != cudaSuccess) return cuda_status(e);
        float ms = 0.f;
        auto span = [&](int a, int b) {
            return cudaEventElapsedTime(&ms, p.ev[a], p.ev[b]) == cudaSuccess ? (double)ms : -1.0;
        };
        times_ms[0] = span(kEvStart, kEvBinned);
        times_ms[1] = span(kEvBinned, kEvRealEnd);
        const bool rc = p.prof_recip;   // the reciprocal branch ran in that evaluation
        times_ms[2] = rc ? span(kEvRecipStart, kEvFwdEnd) : -1.0;
        times_ms[3] = rc ? span(kEvFwdEnd, kEvCoefEnd) : -1.0;
        times_ms[4] = rc ? span(kEvCoefEnd, kEvBackEnd) : -1.0;
        times_ms[5] = span(kEvRealEnd, kEvFinal);
        times_ms[6] = span(kEvStart, kEvFinal);
        times_ms[7] = rc ? span(kEvRecipStart, kEvBackEnd) : -1.0;
        times_ms[8] = span(kEvRealStart, kEvRealEnd);
        times_ms[9] = rc && p.prof_bs ? span(kEvBsStart, kEvBsEnd) : -1.0;
        times_ms[10] = span(kEvJoined, kEvFinal);
    }
    return EWALD_OK;
}

extern "C" int ewald_plan_info(ewald_plan_t plan, int64_t info[6])
{
    if (!plan || !info) return EWALD_E_INVAL;
    const Plan &p = plan->p;
    info[0] = p.nc; info[1] = p.w; info[2] = p.nk; info[3] = p.R; info[4] = p.kmax;
    info[5] = p.precision;
    return EWALD_OK;
}

extern "C" int ewald_kset(ewald_plan_t plan, int32_t *m_host, int64_t cap, int64_t *count)
{
    if (!plan) return EWALD_E_INVAL;
    const Plan &p = plan->p;
    if (count) *count = p.nk;
    if (m_host && cap > 0) {
        int64_t m = cap < p.nk ? cap : p.nk;
        cudaError_t e = cudaMemcpy(m_host, p.kset_d, sizeof(int) * 3 * m, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return EWALD_OK;
}

extern "C" int ewald_structure_factor(ewald_plan_t plan, double *S_dev, void *stream)
{
    if (!plan || !S_dev) return EWALD_E_INVAL;
    const Plan &p = plan->p;
    if (p.spme) return EWALD_E_UNSUPPORTED;
    return cuda_status(cudaMemcpyAsync(S_dev, p.S_d, sizeof(double) * 2 * p.nk,
                                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

extern "C" int ewald_cell_sort(ewald_plan_t plan, int32_t *key_dev, int32_t *perm_dev, void *stream)
{
    if (!plan) return EWALD_E_INVAL;
    const Plan &p = plan->p;
    const int64_t n = p.ws.cap_n;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (key_dev && n) e = cudaMemcpyAsync(key_dev, p.ws.key, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && perm_dev && n)
        e = cudaMemcpyAsync(perm_dev, p.ws.perm, sizeof(int) * n, cudaMemcpyDeviceToDevice, st);
    return cuda_status(e);
}

// ---- tuner --------------------------------------------------------------------------------

extern "C" int ewald_tune(int64_t n, double L, double tol, double *r_c, double *beta, int *k_max)
{
    if (!r_c || !beta || !k_max || n < 2 || !(L > 0) || !(tol > 1e-15) || !(tol < 0.1))
        return EWALD_E_INVAL;
    // Both truncation errors fall as exp(-p^2), p = beta r_c = pi k_max / (beta L); the
    // relative RMS force error of dense ionic systems is close to exp(-p^2) itself.
    const double p = sqrt(-log(tol));
    double rc = *r_c;
    if (!(rc > 0)) {
        // Cost per particle, calibrated on GB300 with the EWALD_MIXED path (262,144- and
        // 2,097,152-ion systems, each part timed alone): real space ~1.3e-11 s per r_c^3 rho,
        // the two reciprocal products ~1.1e-13 s per k_max^3, k_max = p^2 L / (pi r_c).  Pick
        // the r_c <= L/2 that minimises the sum on a grid (where the two parts cost about the
        // same, which also balances the two streams they run on).
        const double rho = n / (L * L * L);
        const double c_pair = 1.3e-11, c_mode = 1.1e-13;
        double best = 1e300, best_rc = 0.5 * L;
        for (int t = 1; t <= 400; ++t) {
            double x = 0.5 * L * t / 400.0;
            if (x < 1e-3) continue;
            double km = p * p * L / (kPi * x);
            double cost = c_pair * x * x * x * rho + c_mode * km * km * km;
            if (cost < best) { best = cost; best_rc = x; }
        }
        rc = best_rc;
    }
    if (rc > 0.5 * L) return EWALD_E_CUTOFF;
    const double b = p / rc;
    int km = (int)ceil(p * b * L / kPi);
    if (km < 1) km = 1;
    if (km > 127) return EWALD_E_UNSUPPORTED;
    *r_c = rc;
    *beta = b;
    *k_max = km;
    return EWALD_OK;
}

extern "C" const char *ewald_strerror(int status)
{
    switch (status) {
    case EWALD_OK: return "EWALD_OK";
    case EWALD_PENDING: return "EWALD_PENDING";
    case EWALD_E_INVAL: return "EWALD_E_INVAL: invalid argument";
    case EWALD_E_NONNEUTRAL: return "EWALD_E_NONNEUTRAL: the system is not charge neutral";
    case EWALD_E_CUTOFF: return "EWALD_E_CUTOFF: r_c must satisfy 0 < r_c <= L/2";
    case EWALD_E_NOMEM: return "EWALD_E_NOMEM: out of device memory or over the budget";
    case EWALD_E_CUDA: return "EWALD_E_CUDA: a CUDA call failed";
    case EWALD_E_TIMEOUT: return "EWALD_E_TIMEOUT: a bounded wait gave up";
    case EWALD_E_BUSY: return "EWALD_E_BUSY: no free slot or the queue is full";
    case EWALD_E_NOTFOUND: return "EWALD_E_NOTFOUND: unknown ticket";
    case EWALD_E_NONFINITE: return "EWALD_E_NONFINITE: a position or charge is not finite";
    case EWALD_E_UNSUPPORTED: return "EWALD_E_UNSUPPORTED: parameters outside this build";
    default: return "EWALD_E_UNKNOWN";
    }
}
