/*
 * Random sequential insertion of hard-core points in a periodic cube (input generation
 * only: no Ewald arithmetic).
 *
 * Candidates arrive in a fixed stream (drawn by the caller from a seeded generator); each
 * one is accepted when no accepted point lies closer than the hard core under the periodic
 * minimum image, and rejected otherwise, strictly in stream order.  Accepted points are kept
 * in a grid of g^3 cells of side L / g >= hard core, one linked list per cell, so that a
 * candidate is compared only with the points of its own and the 26 neighbouring cells
 * (g >= 3); for g < 3 every accepted point is compared.
 *
 * Build with -ffp-contract=off: the accept/reject decisions must be the same on every host,
 * so no multiply-add may be fused differently by one compiler than by another.
 */
#include <math.h>
#include <stdint.h>

static int cell_of(double x, double L, int g)
{
    int c = (int)(x / L * g);
    if (c < 0) c = 0;
    if (c >= g) c = g - 1;
    return c;
}

static int wrap_cell(int c, int g)
{
    return c < 0 ? c + g : (c >= g ? c - g : c);
}

/* Minimum image of a difference of two coordinates in [0, L), so d is in (-L, L). */
static double min_image(double d, double L)
{
    return d >= 0.5 * L ? d - L : (d < -0.5 * L ? d + L : d);
}

/*
 * Consume candidates cand[0 .. ncand) (xyz triples in [0, L)) until `count` reaches
 * n_target.  pts [n_target][3] holds the `count` points accepted so far; head [g^3] and
 * next [n_target] are the cell lists (head initialised to -1 by the caller before the first
 * call).  Returns the new count and writes the number of candidates consumed.
 */
int64_t rsa_insert(double L, double hard_core, int g, int64_t n_target, int64_t count,
                   double *pts, int64_t *head, int64_t *next, const double *cand,
                   int64_t ncand, int64_t *consumed)
{
    const double hc2 = hard_core * hard_core;
    int64_t c = 0;
    for (; c < ncand && count < n_target; ++c) {
        const double x = cand[3 * c], y = cand[3 * c + 1], z = cand[3 * c + 2];
        int ok = 1;
        if (g >= 3) {
            const int cx = cell_of(x, L, g), cy = cell_of(y, L, g), cz = cell_of(z, L, g);
            int ux[3], uy[3], uz[3];   /* the neighbouring cell indices, wrapped */
            for (int d = 0; d < 3; ++d) {
                ux[d] = wrap_cell(cx + d - 1, g);
                uy[d] = wrap_cell(cy + d - 1, g);
                uz[d] = wrap_cell(cz + d - 1, g);
            }
            for (int dz = 0; dz < 3 && ok; ++dz)
                for (int dy = 0; dy < 3 && ok; ++dy)
                    for (int dx = 0; dx < 3 && ok; ++dx) {
                        for (int64_t p = head[((int64_t)uz[dz] * g + uy[dy]) * g + ux[dx]];
                             p >= 0; p = next[p]) {
                            const double ex = min_image(x - pts[3 * p], L);
                            const double ey = min_image(y - pts[3 * p + 1], L);
                            const double ez = min_image(z - pts[3 * p + 2], L);
                            if (ex * ex + ey * ey + ez * ez < hc2) { ok = 0; break; }
                        }
                    }
        } else {
            for (int64_t p = 0; p < count && ok; ++p) {
                const double ex = min_image(x - pts[3 * p], L);
                const double ey = min_image(y - pts[3 * p + 1], L);
                const double ez = min_image(z - pts[3 * p + 2], L);
                if (ex * ex + ey * ey + ez * ez < hc2) ok = 0;
            }
        }
        if (!ok) continue;
        pts[3 * count] = x;
        pts[3 * count + 1] = y;
        pts[3 * count + 2] = z;
        if (g >= 3) {
            const int64_t key =
                ((int64_t)cell_of(z, L, g) * g + cell_of(y, L, g)) * g + cell_of(x, L, g);
            next[count] = head[key];
            head[key] = count;
        }
        ++count;
    }
    *consumed = c;
    return count;
}
