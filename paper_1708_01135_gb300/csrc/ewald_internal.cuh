// Internal definitions shared by the CUDA translation units of libewald.so.
//
// Notation follows the paper (arXiv 1708.01135, Section 3): N charges q_j at r_j in a cubic
// box of side L; splitting parameter beta (the paper's alpha = beta^2); real-space cutoff
// r_c; reciprocal vectors k = 2 pi m / L with m in Z^3, |m|^2 <= k_max^2.
//
// The reciprocal sum is organised over "rows": every (m_y, m_z) with m_y^2 + m_z^2 <=
// k_max^2 in the half plane (m_z > 0, or m_z = 0 and m_y >= 0), ordered by m_z then m_y.
// Along a row m_x runs over [-k_max, k_max]; the modes of K_half on row r are
// m_x in [-nxmax_r, nxmax_r] (m_x > 0 only on the row (0, 0)), nxmax_r =
// floor(sqrt(k_max^2 - m_y^2 - m_z^2)).  This turns S(k) = sum_j q_j exp(i k.r_j) into the
// matrix product of Eq. 3: S[r, m_x] = sum_j (q_j e^{i(k_y y_j + k_z z_j)}) e^{i k_x x_j}.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ewald.h"

struct ewald_plan;

namespace ew {

constexpr double kPi = 3.14159265358979323846;

// Device status bits, OR-ed into plan->d_status by kernels; translated to ewald_status on
// the host.
enum : int {
    kStNonFinite = 1,
    kStTimeout = 2,
    kStNonNeutral = 4,
    kStBadType = 8,      // a Lennard-Jones type outside [0, ntypes)
    kStRange = 16,       // sum |q| beyond the range of the SPME fixed-point charge mesh
};

// Largest sum |q| for which no point of the SPME fixed-point mesh (2^-36 resolution in a
// signed 64-bit integer) can overflow: every particle adds at most |q| to a point.
constexpr double kSpmeMaxAbsCharge = 67108864.0;   // 2^26

// Row of the reciprocal grid: (m_y, m_z), nxmax, and the offset of its first mode in the
// K_half ordering.
struct RowInfo {
    int my, mz, nxmax, koff;
};

constexpr int kMaxCellsPerSide = 160;   // cells per side of the real-space grid, at most

struct Workspace {
    int64_t cap_n = 0;       // particles the buffers hold
    // capacities of the buffers sized by the cell grid (cells, rows of cells, warp tiles,
    // histogram counters), so that another grid that fits reuses them
    int64_t cap_cells = 0, cap_rows = 0, cap_tiles = 0, cap_hist = 0;
    int nb = 0;              // binning chunks (histogram rows)
    // binning
    int *key = nullptr;          // [n] cell index, caller order
    int *perm = nullptr;         // [n] sorted slot -> caller index
    int *key_sorted = nullptr;   // [n]
    int *hist = nullptr;         // [nb * nrows] per-chunk counts of the rows of cells -> offsets
    int *cell_start = nullptr;   // [ncells + 1]
    int *cell_total = nullptr;   // [nrows] particles per row of cells
    int *row_start = nullptr;    // [nrows + 1]
    int *perm1 = nullptr;        // [n] caller index, sorted by row (binning level 1)
    int *key1 = nullptr;         // [n] cell key, sorted by row (binning level 1)
    int2 *tiles = nullptr;       // [max tiles] (row, first slot) of the cell kernel's warps
    int *tile_off = nullptr;     // [nrows + 1] exclusive offsets; tile_off[nrows] = tiles
    int *unordered = nullptr;    // [1] nonzero when a cell was too full to order by x
    // packed particles (sorted)
    double4_32a *pg = nullptr;       // wrapped global position + q (FP64)
    double4_32a *pl64 = nullptr;     // cell-local position + q (FP64, all-pairs mode only)
    float4 *pl32 = nullptr;      // cell-local position + q (FP32, all-pairs mode only)
    uint4 *pu = nullptr;         // 32-bit fixed-point fractions x/L, y/L, z/L + q (float bits):
                                 // the FP32 cell kernel's records and the tensor-core phases
    // outputs (sorted)
    double *f_real = nullptr;    // [n][3]
    double *phi_real = nullptr;  // [n] real-space potential of every sorted particle
    double *phi_recip = nullptr; // [n] reciprocal-space potential of every sorted particle
    double *f_recip = nullptr;   // [n][3]
    double *e_tile = nullptr;    // [max tiles] per-tile q_i phi_i sums
    double *vir_tile = nullptr;  // [12][max tiles] per-tile real-space virial sums (xx yy zz xy xz
                                 // yz; rows 0-5 Coulomb, 6-11 Lennard-Jones)
    int *type_sorted = nullptr;  // [n] Lennard-Jones types in sorted order
    double *elj_tile = nullptr;  // [max tiles] per-tile Lennard-Jones energies
    double *vir_part = nullptr;  // [6][kVirBlocks] block sums of the reciprocal virial
    double *qpart = nullptr;     // [qblocks][3]: sum q, sum |q|, sum q^2 partials
    // staging for the host-buffer entry point
    double *h_pos = nullptr, *h_q = nullptr, *h_f = nullptr, *h_e = nullptr;
    int64_t cap_host = 0;
    // reciprocal (SIMT paths)
    void *tabX = nullptr, *tabY = nullptr, *tabZ = nullptr;   // phase tables, n-major
    void *spart = nullptr;       // forward partials
    size_t spart_bytes = 0;
    void *gmat = nullptr;        // back-scatter coefficient matrix
    size_t gmat_bytes = 0;
    int nks = 0;                 // forward K splits
};

struct Plan {
    int device = 0;
    int num_sms = 148;           // streaming multiprocessors of the plan's device
    double L = 0, beta = 0, rc = 0;
    int kmax = 0;
    int precision = 0;
    // cells
    int nc = 1;          // cells per side
    int w = 0;           // stencil half-width in cells (0: all pairs, minimum image)
    int ncells = 1;
    double cell_side = 0;
    int real_tile = 2;           // lanes per target of the real-space cell kernel (2 or 4)
    bool near_df = false;        // FP32 kernel: near Coulomb pairs in double-float arithmetic
    // Lennard-Jones pairs fused into the real-space kernel (off when lj_ntypes == 0)
    int lj_ntypes = 0;
    const int *lj_type = nullptr;    // caller-owned [n] types, caller order
    double *lj_tab_d = nullptr;      // [T][T][4]: sigma^2, 4 eps, 24 eps, 0
    // reciprocal rows
    int R = 0;
    int64_t nk = 0;
    std::vector<RowInfo> rows_h;
    RowInfo *rows_d = nullptr;
    int *fperm_d = nullptr;      // [R] forward order (decreasing n_x,max) -> row index (tensor-core forward)
    int *kset_d = nullptr;       // [nk][3]
    double *S_d = nullptr;       // [nk][2] last structure factor
    double *g_d = nullptr;       // [nk] g(k) = 4 pi exp(-k^2 / (4 beta^2)) / (V k^2), K_half order
    double *e_recip_part = nullptr;  // partial reciprocal energies [e_recip_count]
    int e_recip_count = 0;       // entries of e_recip_part summed by the finalize step
    double *energy_d = nullptr;  // [4] internal energies for the synchronous entry points
    int cap_R = 0;               // rows the row-sized arrays hold
    int64_t cap_nk = 0;          // modes the k-sized arrays hold
    int *d_status = nullptr;
    int *h_status = nullptr;     // pinned mirror
    cudaStream_t last_stream = nullptr;
    cudaStream_t side_stream = nullptr;  // reciprocal branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // CUDA-graph replay of repeated evaluations (see evaluate): the graph runs on the plan's
    // own stream, ordered after and before the caller's stream by two events
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t ev_gin = nullptr, ev_gout = nullptr;
    cudaGraphExec_t gexec = nullptr;
    struct EvalKey {
        int64_t n = -1;
        const void *pos = nullptr, *q = nullptr;
        void *forces = nullptr, *energy = nullptr, *phi = nullptr, *vir = nullptr;
        int parts = 0;
        bool clear = false;
        bool operator==(const EvalKey &o) const
        {
            return n == o.n && pos == o.pos && q == o.q && forces == o.forces &&
                   energy == o.energy && phi == o.phi && vir == o.vir && parts == o.parts &&
                   clear == o.clear;
        }
    };
    EvalKey gkey, last_key;      // key of the captured graph; key of the previous evaluation
    int g_launches = 0;
    Workspace ws;
    // tensor-core path state (allocated lazily)
    void *tc = nullptr;
    // smooth particle-mesh Ewald state (ewald_set_spme); the reciprocal part uses it when set
    void *spme = nullptr;
    // profiling: events at stage boundaries (see ewald_profile), kernel launch counter
    bool prof = false;
    bool prof_valid = false;
    bool prof_bs = false;        // the back-scatter kernel events were recorded
    bool prof_recip = false;     // the reciprocal branch's events were recorded
    cudaEvent_t ev[12] = {};
    int launches = 0;
};

// Stage boundary events (recorded only while profiling is on).
enum : int {
    kEvStart = 0, kEvBinned = 1, kEvRealEnd = 2, kEvRecipStart = 3, kEvFwdEnd = 4,
    kEvCoefEnd = 5, kEvBackEnd = 6, kEvFinal = 7, kEvRealStart = 8, kEvBsStart = 9,
    kEvBsEnd = 10, kEvJoined = 11,
};
inline void prof_mark(Plan &p, int which, cudaStream_t st)
{
    if (p.prof) cudaEventRecord(p.ev[which], st);
}

// ---- launchers (each returns cudaError_t of the launch) --------------------------------

// a1-a3: wrap, cell keys, stable counting sort, cell offsets, packing.
cudaError_t launch_binning(Plan &p, int64_t n, const double *pos, const double *q,
                           cudaStream_t st);
// a4: real-space pairs into ws.f_real / ws.phi_real / ws.e_tile (sorted order), and with
// virial the per-tile virial sums into ws.vir_tile.
cudaError_t launch_real(Plan &p, int64_t n, cudaStream_t st, bool virial);
// One bounded device wait that cannot complete (the timeout path of the staged copies).
cudaError_t launch_wait_probe(Plan &p, cudaStream_t st);
int64_t real_tile_capacity(const Plan &p, int64_t n);   // energy partials (target groups)
int real_tile_size(const Plan &p);          // targets per real-space warp
int real_tile_for(int w, double cell_occupancy);   // lanes per target for a grid (particles per cell)
// x windows of the real-space cell kernel (FP32 records): binning orders every cell by x and
// the kernel cuts each target's candidates to its own x window.  They pay where the rows are
// long (stencil half-width w >= 5: the 262,144- and 2,097,152-ion systems; at w = 3 and 4 the
// searches and the x order cost what the dropped candidates save), and every x displacement
// a window test takes must stay below L/2 in magnitude (reach + one cell side < L/2).
inline bool use_xwin(const Plan &p)
{
    return p.precision != EWALD_FP64 && p.w >= 5 &&
           p.rc * 1.00001 + p.cell_side < 0.5 * p.L * (1.0 - 1e-6);
}
// a5-a8 on CUDA cores (FP64 or FP32): S(k), energy, back-scatter into ws.f_recip.
cudaError_t launch_recip_simt(Plan &p, int64_t n, cudaStream_t st);
size_t recip_simt_bytes(const Plan &p, int64_t n);
cudaError_t alloc_recip_simt(Plan &p, int64_t n);
void free_recip_simt(Plan &p);
// a5-a8 on the tcgen05 tensor cores (split FP16/BF16 operands).
cudaError_t launch_recip_tc(Plan &p, int64_t n, cudaStream_t st);
// a5 column operand of the forward product; launched before the fork, so that the forward
// product is ready to start together with the real-space kernel and takes its SMs first
cudaError_t launch_recip_tc_operands(Plan &p, int64_t n, cudaStream_t st);
cudaError_t alloc_recip_tc(Plan &p, int64_t n);
size_t recip_tc_bytes(const Plan &p, int64_t n);
int recip_tc_energy_parts(const Plan &p);   // entries of the partial reciprocal energies
void free_recip_tc(Plan &p);
// Smooth particle-mesh Ewald reciprocal part into ws.f_recip / ws.phi_recip, its energy
// partials (spme_energy_parts) and virial partials (spme_virial_parts).
int spme_set(Plan &p, int K, int order);     // K = 0: back to the classical sum
void spme_free(Plan &p);
cudaError_t launch_recip_spme(Plan &p, int64_t n, cudaStream_t st);
const double *spme_energy_parts(const Plan &p, int *count);   // [count] energy partials
const double *spme_virial_parts(const Plan &p, int *count);   // [6][count] virial partials
size_t spme_bytes(const Plan &p);
// One whole evaluation on `st` (grows the workspaces for n first; n > 0).  With
// clear_status false the plan's device status keeps the bits of earlier evaluations, so that
// a sequence of evaluations reports every failure at the next ewald_status_sync.
// phi (optional, [n] caller order) receives the potentials; vir (optional, [4][9]) the
// virial tensors of the real, reciprocal and self parts and their total.
cudaError_t evaluate(Plan &p, int64_t n, const double *pos, const double *q, double *forces,
                     double *energy_dev, int parts, cudaStream_t st, bool clear_status,
                     double *phi = nullptr, double *vir = nullptr);

// Library memory pool (stream-ordered, retains freed memory for reuse).
cudaError_t pool_alloc(void **ptr, size_t bytes, cudaStream_t st);
// The kernel may use up to the device's opt-in dynamic shared memory (set once, never lowered);
// max_dynamic (optional) receives that size.
cudaError_t smem_optin(const void *func, size_t *max_dynamic = nullptr);
void pool_free(void *ptr, cudaStream_t st);

// Host-side plan set-up shared by ewald_create and the server: validates the parameters,
// chooses the cell grid and enumerates the reciprocal rows (no device work).
int plan_setup_host(Plan &p, double L, double beta, double rc, int kmax, int precision);

// Re-parameterise an existing plan (keeps its streams and, when the grid and k-set shapes
// are unchanged, its workspaces).
int plan_reconfigure(struct ::ewald_plan *h, double L, double beta, double rc, int kmax,
                     int precision);

// Footprint of a plan's workspaces for n particles (serving admission).
size_t plan_footprint(const Plan &p, int64_t n);

// Blocks of the reciprocal virial reduction (each sums a fixed stride of the modes).
constexpr int kVirBlocks = 128;

// Bounded spin limit for mbarrier waits inside kernels (iterations of try_wait).
constexpr long long kSpinLimit = 1ll << 26;

}  // namespace ew

// Opaque handle of the C ABI (ewald_plan_t points to one of these).
struct ewald_plan {
    ew::Plan p;
};
