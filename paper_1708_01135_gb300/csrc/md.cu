// ewald_md: velocity-Verlet time stepping driven by the Ewald forces.
//
// The paper computes the Ewald forces once per MD time step (Section 2.1) and benchmarks
// the time per step of an NaCl system (Section 4).  This file runs such a loop on the
// device: every step is a half kick, a drift, one full evaluation (the same pipeline as
// ewald_compute_async) and a second half kick that also forms the kinetic energy.  Nothing
// synchronises with the host inside the loop; per-step energies go to a caller-owned device
// log.
//
// The kick/drift kernels are elementwise over the 3n coordinates (24 bytes of position,
// velocity and force per coordinate triple read, 16 written); the kinetic energy is a
// block-partial sum in a fixed order followed by a one-block fixed-order sum, so the energy
// log is bit-reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace {

constexpr int kThreads = 256;

// v <- v + hdt F / m;  x <- x + dt v, one coordinate per thread.
__global__ void k_md_kick_drift(int64_t n3, double *__restrict__ pos, double *__restrict__ vel,
                                const double *__restrict__ f, const double *__restrict__ mass,
                                double hdt, double dt)
{
    const int64_t t = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (t >= n3) return;
    const double w = mass ? hdt / mass[t / 3] : hdt;
    const double v = fma(w, f[t], vel[t]);
    vel[t] = v;
    pos[t] = fma(dt, v, pos[t]);
}

// v <- v + hdt F / m for one particle per thread, and the block's partial of
// 1/2 sum m |v|^2 (fixed tree over the block) into ke_part[block].
__global__ void k_md_kick_ke(int64_t n, double *__restrict__ vel, const double *__restrict__ f,
                             const double *__restrict__ mass, double hdt,
                             double *__restrict__ ke_part)
{
    __shared__ double red[kThreads];
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        const double m = mass ? mass[i] : 1.0;
        const double w = hdt / m;
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = fma(w, f[3 * i + a], vel[3 * i + a]);
            if (hdt != 0.0) vel[3 * i + a] = v;
            s = fma(v, v, s);
        }
        ke = 0.5 * m * s;
    }
    red[threadIdx.x] = ke;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) ke_part[blockIdx.x] = red[0];
}

// One block: E_kin = sum of the block partials (each thread a contiguous slice, then a
// fixed tree); rec = (the four energies of this step's evaluation, E_kin, E_pot + E_kin).
__global__ void k_md_record(int nb, const double *__restrict__ ke_part,
                            const double *__restrict__ epot, double *__restrict__ rec)
{
    __shared__ double red[kThreads];
    const int t = threadIdx.x;
    const int per = (nb + kThreads - 1) / kThreads;
    const int b = t * per, e = min(nb, b + per);
    double s = 0.0;
    for (int i = b; i < e; ++i) s += ke_part[i];
    red[t] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    if (t == 0) {
        for (int i = 0; i < 4; ++i) rec[i] = epot[i];
        rec[EWALD_MD_KIN] = red[0];
        rec[EWALD_MD_TOTAL] = epot[EWALD_MD_POT] + red[0];
    }
}

__global__ void k_md_zero(double *__restrict__ x, int64_t m)
{
    const int64_t t = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (t < m) x[t] = 0.0;
}

}  // namespace

extern "C" int ewald_md(ewald_plan_t plan, int64_t n, double *pos, double *vel, const double *q,
                        const double *mass, double dt, int steps, double *forces,
                        double *energy_log, void *stream)
{
    if (!plan || n < 0 || n > (int64_t)INT32_MAX / 4 || steps < 0) return EWALD_E_INVAL;
    if (!(dt > 0) || !isfinite(dt)) return EWALD_E_INVAL;
    if (n > 0 && (!pos || !vel || !q || !forces)) return EWALD_E_INVAL;
    ew::Plan &p = plan->p;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const int64_t nrec = (int64_t)(steps + 1) * EWALD_MD_RECORD;
    if (n == 0) {
        if (energy_log)
            k_md_zero<<<(unsigned)((nrec + kThreads - 1) / kThreads), kThreads, 0, st>>>(energy_log, nrec);
        p.last_stream = st;
        return cudaGetLastError() == cudaSuccess ? EWALD_OK : EWALD_E_CUDA;
    }
    const int nb = (int)((n + kThreads - 1) / kThreads);
    // scratch: [nb] kinetic-energy partials, the energies of the current evaluation (a fixed
    // buffer, so that repeated evaluations replay one captured graph), one record if no log
    double *scratch = nullptr;
    if ((e = ew::pool_alloc((void **)&scratch, sizeof(double) * (nb + 4 + EWALD_MD_RECORD), st)) != cudaSuccess)
        return EWALD_E_NOMEM;
    double *ke_part = scratch, *epot = scratch + nb;
    auto record = [&](int s) {
        return energy_log ? energy_log + (int64_t)s * EWALD_MD_RECORD : scratch + nb + 4;
    };
    const unsigned gb3 = (unsigned)((3 * n + kThreads - 1) / kThreads);
    const double hdt = 0.5 * dt;
    int status = EWALD_OK;
    // initial forces and energies; the device status collects every evaluation of the run
    e = cudaMemsetAsync(p.d_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = ew::evaluate(p, n, pos, q, forces, epot, EWALD_PART_ALL, st, false);
    if (e == cudaSuccess) {
        k_md_kick_ke<<<nb, kThreads, 0, st>>>(n, vel, forces, mass, 0.0, ke_part);
        k_md_record<<<1, kThreads, 0, st>>>(nb, ke_part, epot, record(0));
        e = cudaGetLastError();
    }
    for (int s = 1; s <= steps && e == cudaSuccess; ++s) {
        k_md_kick_drift<<<gb3, kThreads, 0, st>>>(3 * n, pos, vel, forces, mass, hdt, dt);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        e = ew::evaluate(p, n, pos, q, forces, epot, EWALD_PART_ALL, st, false);
        if (e != cudaSuccess) break;
        k_md_kick_ke<<<nb, kThreads, 0, st>>>(n, vel, forces, mass, hdt, ke_part);
        k_md_record<<<1, kThreads, 0, st>>>(nb, ke_part, epot, record(s));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) status = (e == cudaErrorMemoryAllocation) ? EWALD_E_NOMEM : EWALD_E_CUDA;
    ew::pool_free(scratch, st);
    p.last_stream = st;
    return status;
}
