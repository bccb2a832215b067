/*
 * Plain FP64 CPU Ewald summation: the oracle that the CUDA path is checked against.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or loads this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (paper: Sections 3.1-3.2, Eqs. 2-4, Listing 1, Algorithms 1-2):
 *   N point charges q_j at r_j in a periodic cubic box of side L, Gaussian units
 *   (Coulomb constant 1).  The splitting parameter is passed as beta (1/length); the
 *   paper's Gaussian exponent is alpha = beta^2, so erfc(sqrt(alpha) r) = erfc(beta r).
 *
 *   E_real  = 1/2 sum_i sum_{j, n: 0 < |r_i - r_j - nL| < r_c}  q_i q_j erfc(beta d)/d
 *             (Section 3.1.1 and Eq. 4; the 1/2 of Listing 1 counts every pair once)
 *   F_i^real = sum_{j, n} q_i q_j (d_vec/d^2) [erfc(beta d)/d + 2 beta/sqrt(pi) exp(-beta^2 d^2)]
 *             with d_vec = r_i - r_j - nL  (Eq. 4, second line)
 *   S(k)    = sum_j q_j exp(i k.r_j),  k = 2 pi m / L,  m in Z^3  (Section 3.1.2; the paper's
 *             rho_hat_k of Eq. 3 is conj(S(k)) without the Gaussian factor)
 *   E_recip = 1/2 sum_{k != 0, |m| <= kmax} g(k) |S(k)|^2,
 *             g(k) = 4 pi exp(-k^2 / (4 beta^2)) / (V k^2)   (C_k of Eq. 3, V = L^3)
 *           = sum_{k in K_half} g(k) |S(k)|^2  over the half space (see kset_half)
 *   F_i^recip = q_i sum_{k in K_half} 2 g(k) k Im(exp(i k.r_i) conj S(k))   (Algorithm 2,
 *             the -i k C_k A q rho_hat update, with k and -k paired so the result is real)
 *   phi_i^recip = sum_{k in K_half} 2 g(k) Re(exp(i k.r_i) conj S(k))       (Algorithm 2, u)
 *   E_self  = -beta/sqrt(pi) sum_i q_i^2    (Section 3.2.2: computed once; formula not
 *             printed in the paper, taken as the standard Gaussian self-interaction)
 *
 * The k = 0 term is dropped (neutral systems, footnote of Section 3.1.2), which is the
 * conducting ("tin-foil") boundary condition.  The reciprocal cutoff is the sphere
 * |m|^2 <= kmax^2 (Algorithm 1 loops over |k| < k_c; this library states the cutoff as an
 * integer radius kmax, inclusive).
 *
 * Every structure factor is evaluated with direct cos/sin per (k, particle): no phase
 * recurrence, no matrix product.  The only parallelism is OpenMP over independent outputs
 * (one k, or one particle, per iteration); every sum over an index runs in index order, and
 * global energies are summed serially after the parallel loop.
 *
 * Parity pins (all in tests/test_oracle.py): Madelung constants of rock-salt and CsCl,
 * invariance of the total energy under beta at converged cutoffs, sum of forces = 0,
 * central finite differences of the energy, brute-force image sums of tiny neutral cells
 * (ewo_coulomb_cube), the exactly known S(k) of an unjittered rock-salt lattice,
 * lattice-point counts for the k-set, equality of the cell-list real-space sum
 * (ewo_real_cells) with the all-pairs one (ewo_real), and for the virial tensors: central
 * finite differences of the energies under strain, the Coulomb virial identity
 * tr W = E_total, invariance of W under beta, and the isotropic W = E/3 of rock-salt;
 * for the Lennard-Jones pairs (ewo_lj): the minimum and zero of the pair potential, the
 * simple-cubic lattice sum of (sigma/d)^12, finite differences of the energy under
 * displacement and strain, and invariance under a relabelling of the types.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define EWO_PI 3.14159265358979323846

/* Periodic wrap into [0, L): x - L floor(x / L); a result equal to L (rounding of a tiny
 * negative x) is mapped to 0. */
static double wrap1(double x, double L)
{
    double w = x - L * floor(x / L);
    return (w >= L) ? 0.0 : w;
}

int ewo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ewo_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * Half-space k set K_half: integer m = (mx, my, mz) != 0 with mx^2 + my^2 + mz^2 <= kmax^2
 * and (mz > 0) or (mz == 0 and my > 0) or (mz == 0 and my == 0 and mx > 0).
 * Exactly one of every pair {m, -m} is in the set, so sums over all k != 0 of terms that
 * are even in k equal twice the sum over K_half (the pairing behind Algorithm 1's
 * quadrant ordering, Section 4.2).
 * Order: mz ascending, then my ascending, then mx ascending.
 * Writes up to `cap` triples into m_out (if non-NULL) and returns the set size.
 */
int64_t ewo_kset_half(int kmax, int32_t *m_out, int64_t cap)
{
    int64_t count = 0;
    const int64_t k2max = (int64_t)kmax * kmax;
    for (int mz = 0; mz <= kmax; ++mz)
        for (int my = -kmax; my <= kmax; ++my)
            for (int mx = -kmax; mx <= kmax; ++mx) {
                int64_t m2 = (int64_t)mx * mx + (int64_t)my * my + (int64_t)mz * mz;
                if (m2 == 0 || m2 > k2max) continue;
                int in_half = (mz > 0) || (mz == 0 && my > 0) || (mz == 0 && my == 0 && mx > 0);
                if (!in_half) continue;
                if (m_out && count < cap) {
                    m_out[3 * count + 0] = mx;
                    m_out[3 * count + 1] = my;
                    m_out[3 * count + 2] = mz;
                }
                ++count;
            }
    return count;
}

/*
 * Real-space part (Section 3.1.1, Eq. 4, Listing 1) for the target particles `sub`
 * (all particles when sub == NULL, nsub ignored).
 *   phi_out[t]  = sum_{j,n} q_j erfc(beta d)/d                    (may be NULL)
 *   F_out[t]    = q_i sum_{j,n} q_j (d_vec/d^2)[erfc(beta d)/d + 2 beta/sqrt(pi) e^{-beta^2 d^2}]
 *   *e_real     = 1/2 sum_t q_i phi_i   (summed serially in target order; may be NULL)
 * Pairs are counted when 0 < d < r_c (strict, as Listing 1's mask).  For r_c <= L/2 only the
 * nearest image along every axis can lie inside the cutoff, so that image is taken directly;
 * otherwise every shift n with |n_a| <= ceil(r_c / L) is visited (including the particle's
 * own images, which add energy but no net force).  With force_images != 0 the image loop is
 * taken whatever r_c is: for r_c <= L/2 it visits the 27 shifts |n_a| <= 1 and keeps those
 * within r_c, which is the same sum as the minimum image term by term (the tests compare
 * the two branches this way).
 */
void ewo_real(int64_t n, const double *pos, const double *q, double L, double beta, double rc,
              int64_t nsub, const int64_t *sub, double *F_out, double *phi_out, double *e_real,
              int force_images)
{
    const int64_t nt = sub ? nsub : n;
    const double rc2 = rc * rc;
    const double two_beta_rpi = 2.0 * beta / sqrt(EWO_PI);
    const int min_image = (rc <= 0.5 * L) && !force_images;
    const int ms = (int)ceil(rc / L);
    /* phi is needed for the energy even when the caller does not want it */
    double *phi_tmp = phi_out;
    if (!phi_tmp && e_real) phi_tmp = (double *)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(double));

    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = sub ? sub[t] : t;
        const double xi = wrap1(pos[3 * i + 0], L);
        const double yi = wrap1(pos[3 * i + 1], L);
        const double zi = wrap1(pos[3 * i + 2], L);
        double fx = 0.0, fy = 0.0, fz = 0.0, phi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double dx0 = xi - wrap1(pos[3 * j + 0], L);
            const double dy0 = yi - wrap1(pos[3 * j + 1], L);
            const double dz0 = zi - wrap1(pos[3 * j + 2], L);
            if (min_image) {
                if (j == i) continue;
                const double dx = dx0 - L * round(dx0 / L);
                const double dy = dy0 - L * round(dy0 / L);
                const double dz = dz0 - L * round(dz0 / L);
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (!(d2 < rc2)) continue;
                const double d = sqrt(d2);
                const double e = erfc(beta * d) / d;
                const double s = q[j] * (e + two_beta_rpi * exp(-beta * beta * d2)) / d2;
                phi += q[j] * e;
                fx += s * dx; fy += s * dy; fz += s * dz;
            } else {
                for (int sx = -ms; sx <= ms; ++sx)
                    for (int sy = -ms; sy <= ms; ++sy)
                        for (int sz = -ms; sz <= ms; ++sz) {
                            if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                            const double dx = dx0 - L * sx;
                            const double dy = dy0 - L * sy;
                            const double dz = dz0 - L * sz;
                            const double d2 = dx * dx + dy * dy + dz * dz;
                            if (!(d2 < rc2)) continue;
                            const double d = sqrt(d2);
                            const double e = erfc(beta * d) / d;
                            const double s = q[j] * (e + two_beta_rpi * exp(-beta * beta * d2)) / d2;
                            phi += q[j] * e;
                            fx += s * dx; fy += s * dy; fz += s * dz;
                        }
            }
        }
        if (F_out) {
            F_out[3 * t + 0] = q[i] * fx;
            F_out[3 * t + 1] = q[i] * fy;
            F_out[3 * t + 2] = q[i] * fz;
        }
        if (phi_tmp) phi_tmp[t] = phi;
    }
    if (e_real) {
        double e = 0.0;
        for (int64_t t = 0; t < nt; ++t) e += 0.5 * q[sub ? sub[t] : t] * phi_tmp[t];
        *e_real = e;
    }
    if (phi_tmp != phi_out) free(phi_tmp);
}

/*
 * The same real-space sum through a cell list (the binned pair loop of Section 3.1.1), for
 * systems too large for the all-pairs loop above.  Requires r_c <= L/2 (minimum image) and
 * at least 3 cells per side: the box is cut into nc = floor(L / r_c) cells per side, so that
 * every partner within r_c of a target lies in the target's cell or one of its 26
 * neighbours, and those 27 cells are distinct.  Particles are bucketed by a serial counting
 * pass in index order; a target visits its 27 cells in a fixed order and every particle of a
 * cell in index order.  Outputs as ewo_real.  Returns 0, or -1 when the conditions above do
 * not hold (nothing written).
 */
int ewo_real_cells(int64_t n, const double *pos, const double *q, double L, double beta,
                   double rc, int64_t nsub, const int64_t *sub, double *F_out, double *phi_out,
                   double *e_real)
{
    if (!(rc <= 0.5 * L)) return -1;
    const int64_t nc = (int64_t)floor(L / rc);
    if (nc < 3) return -1;
    const int64_t ncell = nc * nc * nc;
    const int64_t nt = sub ? nsub : n;
    const double rc2 = rc * rc;
    const double two_beta_rpi = 2.0 * beta / sqrt(EWO_PI);
    double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    int64_t *cell = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *member = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    double *phi_tmp = phi_out;
    if (!phi_tmp && e_real) phi_tmp = (double *)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            w[3 * j + a] = wrap1(pos[3 * j + a], L);
            int64_t ca = (int64_t)floor(w[3 * j + a] * (double)nc / L);
            if (ca >= nc) ca = nc - 1;
            c[a] = ca;
        }
        cell[j] = (c[2] * nc + c[1]) * nc + c[0];
        start[cell[j] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < ncell; ++c) fill[c] = start[c];
    for (int64_t j = 0; j < n; ++j) member[fill[cell[j]]++] = j;
    /* positions and charges copied into cell order, so that a cell's members are contiguous */
    double *ws = (double *)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(double));
    for (int64_t s = 0; s < n; ++s) {
        const int64_t j = member[s];
        ws[4 * s + 0] = w[3 * j + 0];
        ws[4 * s + 1] = w[3 * j + 1];
        ws[4 * s + 2] = w[3 * j + 2];
        ws[4 * s + 3] = q[j];
    }

    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = sub ? sub[t] : t;
        const double xi = w[3 * i], yi = w[3 * i + 1], zi = w[3 * i + 2];
        const int64_t ci = cell[i];
        const int64_t cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
        double fx = 0.0, fy = 0.0, fz = 0.0, phi = 0.0;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const int64_t c = (((cz + oz + nc) % nc) * nc + (cy + oy + nc) % nc) * nc
                                      + (cx + ox + nc) % nc;
                    for (int64_t s = start[c]; s < start[c + 1]; ++s) {
                        if (member[s] == i) continue;
                        const double *pj = ws + 4 * s;
                        double dx = xi - pj[0], dy = yi - pj[1], dz = zi - pj[2];
                        dx -= L * round(dx / L);
                        dy -= L * round(dy / L);
                        dz -= L * round(dz / L);
                        const double d2 = dx * dx + dy * dy + dz * dz;
                        if (!(d2 < rc2)) continue;
                        const double d = sqrt(d2);
                        const double e = erfc(beta * d) / d;
                        const double sc = pj[3] * (e + two_beta_rpi * exp(-beta * beta * d2)) / d2;
                        phi += pj[3] * e;
                        fx += sc * dx; fy += sc * dy; fz += sc * dz;
                    }
                }
        if (F_out) {
            F_out[3 * t + 0] = q[i] * fx;
            F_out[3 * t + 1] = q[i] * fy;
            F_out[3 * t + 2] = q[i] * fz;
        }
        if (phi_tmp) phi_tmp[t] = phi;
    }
    if (e_real) {
        double e = 0.0;
        for (int64_t t = 0; t < nt; ++t) e += 0.5 * q[sub ? sub[t] : t] * phi_tmp[t];
        *e_real = e;
    }
    if (phi_tmp != phi_out) free(phi_tmp);
    free(w); free(ws); free(cell); free(start); free(member); free(fill);
    return 0;
}

/*
 * Structure factors over an explicit k list (Section 3.1.2; Algorithm 1 accumulates the
 * conjugate): S[2 t] + i S[2 t + 1] = sum_j q_j (cos(k.r_j) + i sin(k.r_j)), k = 2 pi m_t / L.
 * Direct cos/sin of the full phase per (k, particle).
 */
void ewo_structure_factor(int64_t n, const double *pos, const double *q, double L,
                          int64_t nk, const int32_t *m, double *S)
{
    const double tpl = 2.0 * EWO_PI / L;
    #pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < nk; ++t) {
        const double kx = tpl * m[3 * t + 0], ky = tpl * m[3 * t + 1], kz = tpl * m[3 * t + 2];
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double ph = kx * wrap1(pos[3 * j + 0], L) + ky * wrap1(pos[3 * j + 1], L)
                            + kz * wrap1(pos[3 * j + 2], L);
            re += q[j] * cos(ph);
            im += q[j] * sin(ph);
        }
        S[2 * t + 0] = re;
        S[2 * t + 1] = im;
    }
}

/* g(k) = 4 pi exp(-k^2 / (4 beta^2)) / (V k^2)  (C_k of Eq. 3 with alpha = beta^2). */
static double coef_g(const int32_t *mt, double L, double beta)
{
    const double tpl = 2.0 * EWO_PI / L;
    const double kx = tpl * mt[0], ky = tpl * mt[1], kz = tpl * mt[2];
    const double k2 = kx * kx + ky * ky + kz * kz;
    return 4.0 * EWO_PI * exp(-k2 / (4.0 * beta * beta)) / (L * L * L * k2);
}

/* E_recip = sum_{k in K_half} g(k) |S(k)|^2 (equal to 1/2 sum over all k != 0), summed in
 * list order.  Also returns g per k in g_out when non-NULL. */
double ewo_recip_energy(int64_t nk, const int32_t *m, const double *S, double L, double beta,
                        double *g_out)
{
    double e = 0.0;
    for (int64_t t = 0; t < nk; ++t) {
        const double g = coef_g(m + 3 * t, L, beta);
        if (g_out) g_out[t] = g;
        e += g * (S[2 * t] * S[2 * t] + S[2 * t + 1] * S[2 * t + 1]);
    }
    return e;
}

/*
 * Reciprocal forces and potentials for the target particles (Algorithm 2), given S(k) over
 * a half-space k list:
 *   F_out[t]   = q_i sum_k 2 g(k) k Im(exp(i k.r_i) conj S(k))
 *   phi_out[t] = sum_k 2 g(k) Re(exp(i k.r_i) conj S(k))      (either pointer may be NULL)
 */
void ewo_recip_forces(int64_t n, const double *pos, const double *q, double L, double beta,
                      int64_t nk, const int32_t *m, const double *S,
                      int64_t nsub, const int64_t *sub, double *F_out, double *phi_out)
{
    const int64_t nt = sub ? nsub : n;
    const double tpl = 2.0 * EWO_PI / L;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t i = sub ? sub[t] : t;
        const double xi = wrap1(pos[3 * i + 0], L);
        const double yi = wrap1(pos[3 * i + 1], L);
        const double zi = wrap1(pos[3 * i + 2], L);
        double fx = 0.0, fy = 0.0, fz = 0.0, phi = 0.0;
        for (int64_t u = 0; u < nk; ++u) {
            const double kx = tpl * m[3 * u + 0], ky = tpl * m[3 * u + 1], kz = tpl * m[3 * u + 2];
            const double g2 = 2.0 * coef_g(m + 3 * u, L, beta);
            const double ph = kx * xi + ky * yi + kz * zi;
            const double c = cos(ph), s = sin(ph);
            const double sr = S[2 * u], si = S[2 * u + 1];
            /* exp(i ph) * conj(S) = (c + i s)(sr - i si) */
            const double re = c * sr + s * si;
            const double im = s * sr - c * si;
            phi += g2 * re;
            fx += g2 * kx * im; fy += g2 * ky * im; fz += g2 * kz * im;
        }
        if (F_out) {
            F_out[3 * t + 0] = q[i] * fx;
            F_out[3 * t + 1] = q[i] * fy;
            F_out[3 * t + 2] = q[i] * fz;
        }
        if (phi_out) phi_out[t] = phi;
    }
}

/*
 * Real-space virial tensor: the strain derivative W_ab = -dE_real/d(eps_ab) of the real-space
 * energy of Section 3.1.1 when every separation d_vec of Eq. 4 is strained to (1 + eps) d_vec
 * at fixed beta.  With psi(d) = -d/dd [erfc(beta d)/d] = erfc(beta d)/d^2 +
 * 2 beta/sqrt(pi) exp(-beta^2 d^2)/d (the radial factor of Eq. 4's force),
 *   W_ab = 1/2 sum_i sum_{j,n} q_i q_j psi(d) d_a d_b / d,   d_vec = r_i - r_j - nL,
 * i.e. 1/2 sum over ordered pairs of d_a F_b with F the pair force of Eq. 4.  The pairs and
 * images are those of ewo_real (strict 0 < d < r_c).  W_out[3 a + b], row-major.  Each target
 * accumulates its own row in parallel; the rows are added serially in target order.
 */
void ewo_virial_real(int64_t n, const double *pos, const double *q, double L, double beta,
                     double rc, double *W_out)
{
    const double rc2 = rc * rc;
    const double two_beta_rpi = 2.0 * beta / sqrt(EWO_PI);
    const int min_image = (rc <= 0.5 * L);
    const int ms = (int)ceil(rc / L);
    double *rows = (double *)calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));

    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        const double xi = wrap1(pos[3 * i + 0], L);
        const double yi = wrap1(pos[3 * i + 1], L);
        const double zi = wrap1(pos[3 * i + 2], L);
        double w[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            const double dx0 = xi - wrap1(pos[3 * j + 0], L);
            const double dy0 = yi - wrap1(pos[3 * j + 1], L);
            const double dz0 = zi - wrap1(pos[3 * j + 2], L);
            const int lo = min_image ? 0 : -ms, hi = min_image ? 0 : ms;
            for (int sx = lo; sx <= hi; ++sx)
                for (int sy = lo; sy <= hi; ++sy)
                    for (int sz = lo; sz <= hi; ++sz) {
                        if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                        double d[3] = {dx0 - L * sx, dy0 - L * sy, dz0 - L * sz};
                        if (min_image)
                            for (int a = 0; a < 3; ++a) d[a] -= L * round(d[a] / L);
                        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(d2 < rc2)) continue;
                        const double r = sqrt(d2);
                        const double psi = erfc(beta * r) / d2 + two_beta_rpi * exp(-beta * beta * d2) / r;
                        const double c = q[j] * psi / r;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) w[3 * a + b] += c * d[a] * d[b];
                    }
        }
        for (int u = 0; u < 9; ++u) rows[9 * i + u] = 0.5 * q[i] * w[u];
    }
    for (int u = 0; u < 9; ++u) W_out[u] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int u = 0; u < 9; ++u) W_out[u] += rows[9 * i + u];
    free(rows);
}

/*
 * Reciprocal-space virial tensor W_ab = -dE_recip/d(eps_ab) at fixed beta, given S(k) over a
 * half-space k list.  Under the strain the box volume becomes V (1 + tr eps) and every k of
 * Eq. 3 becomes (1 - eps) k while k.r_j, hence S(k), is unchanged; differentiating
 * g(k) = 4 pi exp(-k^2/(4 beta^2)) / (V k^2) gives
 *   W_ab = sum_{k in K_half} g(k) |S(k)|^2 [delta_ab - 2 k_a k_b (1/k^2 + 1/(4 beta^2))],
 * summed serially in list order.  W_out[3 a + b], row-major.
 */
void ewo_virial_recip(int64_t nk, const int32_t *m, const double *S, double L, double beta,
                      double *W_out)
{
    const double tpl = 2.0 * EWO_PI / L;
    for (int u = 0; u < 9; ++u) W_out[u] = 0.0;
    for (int64_t t = 0; t < nk; ++t) {
        const double k[3] = {tpl * m[3 * t + 0], tpl * m[3 * t + 1], tpl * m[3 * t + 2]};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double e = coef_g(m + 3 * t, L, beta) * (S[2 * t] * S[2 * t] + S[2 * t + 1] * S[2 * t + 1]);
        const double c = 2.0 * (1.0 / k2 + 1.0 / (4.0 * beta * beta));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                W_out[3 * a + b] += e * ((a == b ? 1.0 : 0.0) - c * k[a] * k[b]);
    }
}

/*
 * Short-range Lennard-Jones pairs, the repulsion that the paper's NaCl benchmark adds to
 * the Coulomb sum (Section 4; its force-field parameters are not printed).  Every particle
 * has a type t_i in [0, ntypes); eps and sigma are symmetric [ntypes][ntypes] tables.  For
 * 0 < d < r_c (minimum image, the cutoff of the real-space sum) a pair contributes the
 * truncated and shifted potential
 *   u(d) = 4 eps [(sigma/d)^12 - (sigma/d)^6] - 4 eps [(sigma/r_c)^12 - (sigma/r_c)^6],
 * its force on i, F = -du/dd d_vec/d = 24 eps [2 (sigma/d)^12 - (sigma/d)^6] d_vec / d^2,
 * and the strain derivative -du/d(eps_ab) = 1/2 of d_a F_b per ordered pair (as the virial of
 * ewo_virial_real).  Outputs (each may be NULL): F_out [n][3], *e_out = 1/2 sum_i sum_j u,
 * W_out [9] row-major.  Per-target rows in parallel, totals summed serially in index order.
 * Returns 0, or -1 (nothing written) when r_c > L/2 or a type is out of range.
 */
int ewo_lj(int64_t n, const double *pos, const int32_t *type, int ntypes, const double *eps,
           const double *sigma, double L, double rc, double *F_out, double *e_out,
           double *W_out)
{
    if (!(rc <= 0.5 * L) || ntypes < 1) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (type[i] < 0 || type[i] >= ntypes) return -1;
    const double rc2 = rc * rc;
    double *rows = (double *)calloc((size_t)(n > 0 ? n : 1) * 13, sizeof(double));

    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double *row = rows + 13 * i;   /* F[3], u, W[9] */
        const double xi = wrap1(pos[3 * i + 0], L);
        const double yi = wrap1(pos[3 * i + 1], L);
        const double zi = wrap1(pos[3 * i + 2], L);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3] = {xi - wrap1(pos[3 * j + 0], L), yi - wrap1(pos[3 * j + 1], L),
                           zi - wrap1(pos[3 * j + 2], L)};
            for (int a = 0; a < 3; ++a) d[a] -= L * round(d[a] / L);
            const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(d2 < rc2)) continue;
            const int t = type[i] * ntypes + type[j];
            const double e = eps[t], s2 = sigma[t] * sigma[t];
            const double x6 = (s2 / d2) * (s2 / d2) * (s2 / d2);
            const double c6 = (s2 / rc2) * (s2 / rc2) * (s2 / rc2);
            const double f = 24.0 * e * (2.0 * x6 * x6 - x6) / d2;
            row[3] += 4.0 * e * (x6 * x6 - x6) - 4.0 * e * (c6 * c6 - c6);
            for (int a = 0; a < 3; ++a) {
                row[a] += f * d[a];
                for (int b = 0; b < 3; ++b) row[4 + 3 * a + b] += 0.5 * f * d[a] * d[b];
            }
        }
    }
    double e = 0.0, W[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        const double *row = rows + 13 * i;
        if (F_out) for (int a = 0; a < 3; ++a) F_out[3 * i + a] = row[a];
        e += 0.5 * row[3];
        for (int u = 0; u < 9; ++u) W[u] += row[4 + u];
    }
    if (e_out) *e_out = e;
    if (W_out) for (int u = 0; u < 9; ++u) W_out[u] = W[u];
    free(rows);
    return 0;
}

/* E_self = -beta / sqrt(pi) * sum_i q_i^2 (Section 3.2.2, amortised self-energy). */
double ewo_self(int64_t n, const double *q, double beta)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += q[i] * q[i];
    return -beta / sqrt(EWO_PI) * s;
}

/*
 * Brute-force periodic Coulomb sum over whole image cells in a cube of shells
 * (|n_a| <= shells), with the positions exactly as given (NOT wrapped: the cell dipole
 * M = sum_i q_i r_i depends on which image of each charge forms the cell):
 *   E = 1/2 sum_{n} sum_i sum_j' q_i q_j / |r_i - r_j - nL|   (j != i when n = 0)
 *   F_i = q_i sum_{n} sum_j' q_j (r_i - r_j - nL) / |r_i - r_j - nL|^3
 * This is the lattice sum of Section 2.1 taken in one particular (cubic) order; for a
 * neutral cell its limit is the conducting-boundary Ewald energy plus the surface term
 * 2 pi |M|^2 / (3 V) (the conditional convergence discussed in Section 2.1).
 * Sums over the cube in shell order (n by increasing max|n_a|) so that partial results
 * after every shell are available in E_shell[0..shells] when non-NULL.
 */
void ewo_coulomb_cube(int64_t n, const double *pos, const double *q, double L, int shells,
                      double *E_shell, double *F_out)
{
    double e_total = 0.0;
    if (F_out) for (int64_t t = 0; t < 3 * n; ++t) F_out[t] = 0.0;
    for (int s = 0; s <= shells; ++s) {
        double e_shell = 0.0;
        for (int sx = -s; sx <= s; ++sx)
            for (int sy = -s; sy <= s; ++sy)
                for (int sz = -s; sz <= s; ++sz) {
                    int ax = sx < 0 ? -sx : sx, ay = sy < 0 ? -sy : sy, az = sz < 0 ? -sz : sz;
                    int mx = ax > ay ? ax : ay;
                    mx = mx > az ? mx : az;
                    if (mx != s) continue; /* only the cells of this shell */
                    for (int64_t i = 0; i < n; ++i)
                        for (int64_t j = 0; j < n; ++j) {
                            if (s == 0 && i == j) continue;
                            const double dx = pos[3 * i + 0] - pos[3 * j + 0] - L * sx;
                            const double dy = pos[3 * i + 1] - pos[3 * j + 1] - L * sy;
                            const double dz = pos[3 * i + 2] - pos[3 * j + 2] - L * sz;
                            const double d2 = dx * dx + dy * dy + dz * dz;
                            const double d = sqrt(d2);
                            e_shell += 0.5 * q[i] * q[j] / d;
                            if (F_out) {
                                const double f = q[i] * q[j] / (d2 * d);
                                F_out[3 * i + 0] += f * dx;
                                F_out[3 * i + 1] += f * dy;
                                F_out[3 * i + 2] += f * dz;
                            }
                        }
                }
        e_total += e_shell;
        if (E_shell) E_shell[s] = e_total;
    }
}
