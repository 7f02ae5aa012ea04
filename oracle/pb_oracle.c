/*
 * pb_oracle.c -- the ORACLE for the linear Poisson-Boltzmann hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded FP64 C that restates
 * the discretisation and the energy terms of NextGenPB (arXiv 2502.09323) so
 * that the CUDA library can be checked against it.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load this file.  It
 * shares no source, header, table or helper with the CUDA library, and it does
 * not load that library.
 *
 * Units (reduced): lengths in Angstrom, charges in e, potential in kT/e,
 * energies in kT, permittivities relative.  With l_B the vacuum Bjerrum length
 * the equation of Sec. 2.1 (Eq. LPBE) reads
 *     -div(eps grad phi) + eps_s k_D^2 chi_s phi = 4 pi l_B sum_i q_i delta(r - r_i).
 *
 * Discrete system (Sec. 3.1, Eqs. pbe1..matrixequation, with the vertex
 * quadrature that makes the Nedelec mass matrix diagonal):
 *     (G^T W G + C) phi = f
 *   W_e  = eps_e h        edge weight; 1/eps_e is the edge mean of 1/eps,
 *                          which is the weighted harmonic average of Sec. 3.2
 *                          (Eq. WHA) with alpha = inside-length fraction;
 *   C_kk = eps_s k_D^2 h^3 at solvent nodes, 0 at solute nodes;
 *   f_k  = 4 pi l_B sum_i q_i w_k(r_i)  (trilinear weights, Eq. RVop)
 *          + couplings to Dirichlet boundary nodes.
 *
 * Conventions shared with the library's public contract (not its code):
 *   node (i,j,k) has index (k*ny + j)*nx + i and position o + (i,j,k)*h;
 *   edge along axis d from node a has id d*N + a (N = nx*ny*nz);
 *   a node is inside when |x - c|^2 < R^2 for some atom (ties -> solvent),
 *   the squared distance summed as (dx*dx + dy*dy) + dz*dz.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 *
 * Parity unpinned: e_ion_surf (staircase quadrature of the first integral of
 * Eq. energy_ion) has no closed form at finite h; it is pinned only by the
 * convergence of the Kirkwood ionic energy towards its closed form.  The
 * paper's own quadrature of that integral (Sec. 3.3.2: marching cubes through
 * the analytic intersections, vertex rule T_j/3, orc_mc_weights and
 * orc_energy_ion_mc) is pinned by the second-order convergence of the
 * triangulated sphere's area, the exact area of a plane, the solid angle of a
 * union of balls and the Kirkwood ionic energy under refinement.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Units: CODATA 2018 values.                                                 */
/* ------------------------------------------------------------------------ */

/* Vacuum Bjerrum length l_B = e^2 / (4 pi eps0 kB T) in Angstrom and the
 * Debye factor k_D of Sec. 2.1 (k_D^2 = e^2 sum_j z_j^2 rho_j / (eps_s kB T))
 * for a 1:1 salt of ionic strength I mol/L, in 1/Angstrom. */
void orc_units(double temperature_K, double ionic_strength_M, double eps_out,
               double *lB, double *kD)
{
    const double e = 1.602176634e-19;
    const double eps0 = 8.8541878128e-12;
    const double kB = 1.380649e-23;
    const double NA = 6.02214076e23;
    double lb_m = (e * e) / (4.0 * M_PI * eps0 * kB * temperature_K);
    double lb = lb_m * 1e10;
    /* sum_j z_j^2 rho_j = 2 I NA 1e3 per m^3 = 2 I NA 1e-27 per A^3 */
    double kd2 = 4.0 * M_PI * lb * (2.0 * ionic_strength_M * NA * 1e-27) / eps_out;
    *lB = lb;
    *kD = sqrt(kd2);
}

/* ------------------------------------------------------------------------ */
/* Grid placement (perfil, Sec. 2.3 and Sec. 3.4): a cube of side            */
/* fill * extent centred on the molecule's bounding box, extent being the    */
/* largest axis span of the union of [x_i - R_i, x_i + R_i].                 */
/* ------------------------------------------------------------------------ */
void orc_place_grid(const double *atoms, long na, int n, double fill,
                    double origin[3], double *h)
{
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = atoms[d] - atoms[3];
        hi[d] = atoms[d] + atoms[3];
    }
    for (long a = 1; a < na; ++a) {
        const double *p = atoms + 5 * a;
        for (int d = 0; d < 3; ++d) {
            if (p[d] - p[3] < lo[d]) lo[d] = p[d] - p[3];
            if (p[d] + p[3] > hi[d]) hi[d] = p[d] + p[3];
        }
    }
    double ext = 0.0;
    for (int d = 0; d < 3; ++d)
        if (hi[d] - lo[d] > ext) ext = hi[d] - lo[d];
    double L = fill * ext;
    *h = L / (double)(n - 1);
    for (int d = 0; d < 3; ++d)
        origin[d] = 0.5 * (lo[d] + hi[d]) - 0.5 * L;
}

static double coord(const double *o, double h, int d, long i)
{
    return o[d] + (double)i * h;
}

static long clampl(long v, long lo, long hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Index range of nodes along axis d that can lie within radius r of c. */
static void node_range(const int *n, const double *o, double h, int d,
                       double c, double r, long *lo, long *hi)
{
    *lo = clampl((long)floor((c - r - o[d]) / h) - 1, 0, n[d] - 1);
    *hi = clampl((long)ceil((c + r - o[d]) / h) + 1, 0, n[d] - 1);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: eps(r) is eps_m inside the solute (union of atom balls).        */
/* ------------------------------------------------------------------------ */
static int inside_point(const double *atoms, long na, double x, double y, double z)
{
    for (long a = 0; a < na; ++a) {
        const double *p = atoms + 5 * a;
        double dx = x - p[0], dy = y - p[1], dz = z - p[2];
        double d2 = (dx * dx + dy * dy) + dz * dz;
        if (d2 < p[3] * p[3]) return 1;
    }
    return 0;
}

void orc_classify(const int n[3], const double o[3], double h,
                  const double *atoms, long na, uint8_t *inside)
{
    long N = (long)n[0] * n[1] * n[2];
    memset(inside, 0, (size_t)N);
    for (long a = 0; a < na; ++a) {
        const double *p = atoms + 5 * a;
        long lo[3], hi[3];
        for (int d = 0; d < 3; ++d) node_range(n, o, h, d, p[d], p[3], &lo[d], &hi[d]);
        double R2 = p[3] * p[3];
        for (long k = lo[2]; k <= hi[2]; ++k)
            for (long j = lo[1]; j <= hi[1]; ++j)
                for (long i = lo[0]; i <= hi[0]; ++i) {
                    double dx = coord(o, h, 0, i) - p[0];
                    double dy = coord(o, h, 1, j) - p[1];
                    double dz = coord(o, h, 2, k) - p[2];
                    double d2 = (dx * dx + dy * dy) + dz * dz;
                    if (d2 < R2) inside[(k * n[1] + j) * n[0] + i] = 1;
                }
    }
}

/* Brute-force classification of selected nodes (for sampled checks). */
void orc_classify_nodes(const int n[3], const double o[3], double h,
                        const double *atoms, long na, const int64_t *nodes,
                        long count, uint8_t *out)
{
    for (long s = 0; s < count; ++s) {
        long a = nodes[s];
        long i = a % n[0], j = (a / n[0]) % n[1], k = a / ((long)n[0] * n[1]);
        out[s] = (uint8_t)inside_point(atoms, na, coord(o, h, 0, i),
                                       coord(o, h, 1, j), coord(o, h, 2, k));
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: the part of a grid edge that lies in the solute.                */
/* Edge from node a along axis d, parameter t in [0,1], point x_a + t h e_d.  */
/* The ball |x - c| < R meets the line where (u_d + t h)^2 = R^2 - |u_perp|^2 */
/* with u = x_a - c, so t = (-u_d -/+ sqrt(R^2 - |u_perp|^2)) / h.            */
/* The inside fraction alpha is the measure of the union of these intervals  */
/* clipped to [0,1]; for one crossing it is the alpha of Eq. WHA.            */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t id; double t0, t1; } interval;

static int ball_interval(const double *xa, int d, double h, const double *p,
                         double *t0, double *t1)
{
    int e = (d == 0) ? 1 : 0;
    int f = (d == 2) ? 1 : 2;
    double ud = xa[d] - p[d];
    double ue = xa[e] - p[e];
    double uf = xa[f] - p[f];
    double s = p[3] * p[3] - (ue * ue + uf * uf);
    if (!(s > 0.0)) return 0;
    double w = sqrt(s);
    double a0 = (-ud - w) / h;
    double a1 = (-ud + w) / h;
    if (a0 < 0.0) a0 = 0.0;
    if (a1 > 1.0) a1 = 1.0;
    if (!(a1 > a0)) return 0;
    *t0 = a0;
    *t1 = a1;
    return 1;
}

static int cmp_interval(const void *pa, const void *pb)
{
    const interval *a = (const interval *)pa, *b = (const interval *)pb;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    if (a->t0 != b->t0) return a->t0 < b->t0 ? -1 : 1;
    if (a->t1 != b->t1) return a->t1 < b->t1 ? -1 : 1;
    return 0;
}

/* Measure of the union of m intervals sorted by (t0, t1). */
static double union_measure(const interval *v, long m)
{
    if (m == 0) return 0.0;
    double total = 0.0;
    double c0 = v[0].t0, c1 = v[0].t1;
    for (long q = 1; q < m; ++q) {
        if (v[q].t0 <= c1) {
            if (v[q].t1 > c1) c1 = v[q].t1;
        } else {
            total += c1 - c0;
            c0 = v[q].t0;
            c1 = v[q].t1;
        }
    }
    total += c1 - c0;
    return total;
}

static void edge_nodes(const int *n, int64_t id, int *d, long *a, long *b)
{
    long N = (long)n[0] * n[1] * n[2];
    *d = (int)(id / N);
    *a = id % N;
    long stride = (*d == 0) ? 1 : ((*d == 1) ? n[0] : (long)n[0] * n[1]);
    *b = *a + stride;
}

static void node_pos(const int *n, const double *o, double h, long a, double *x)
{
    long i = a % n[0], j = (a / n[0]) % n[1], k = a / ((long)n[0] * n[1]);
    x[0] = coord(o, h, 0, i);
    x[1] = coord(o, h, 1, j);
    x[2] = coord(o, h, 2, k);
}

/* The point r_p where the polarisation charge of a flux edge is placed
 * (Sec. 3.3.1): alpha*h from the inside endpoint towards the outside one.
 * sign = +1 when a is inside and b outside (outward normal +e_d), -1 for the
 * reverse, 0 when both endpoints lie in the same medium (r_p = midpoint). */
static void edge_point(const int *n, const double *o, double h, int64_t id,
                       double alpha, int ina, int inb, double *rp, int *sign)
{
    int d;
    long a, b;
    edge_nodes(n, id, &d, &a, &b);
    double xa[3], xb[3];
    node_pos(n, o, h, a, xa);
    node_pos(n, o, h, b, xb);
    rp[0] = xa[0];
    rp[1] = xa[1];
    rp[2] = xa[2];
    if (ina && !inb) {
        rp[d] = xa[d] + alpha * h;
        *sign = 1;
    } else if (!ina && inb) {
        rp[d] = xb[d] - alpha * h;
        *sign = -1;
    } else {
        rp[d] = xa[d] + 0.5 * h;
        *sign = 0;
    }
}

/* Brute-force alpha for selected edges (all atoms, for sampled checks). */
void orc_edge_alpha(const int n[3], const double o[3], double h,
                    const double *atoms, long na, const int64_t *ids, long count,
                    double *alpha)
{
    interval *buf = (interval *)malloc(sizeof(interval) * (size_t)(na > 0 ? na : 1));
    for (long s = 0; s < count; ++s) {
        int d;
        long a, b;
        edge_nodes(n, ids[s], &d, &a, &b);
        double xa[3];
        node_pos(n, o, h, a, xa);
        long m = 0;
        for (long q = 0; q < na; ++q) {
            double t0, t1;
            if (ball_interval(xa, d, h, atoms + 5 * q, &t0, &t1)) {
                buf[m].id = ids[s];
                buf[m].t0 = t0;
                buf[m].t1 = t1;
                ++m;
            }
        }
        qsort(buf, (size_t)m, sizeof(interval), cmp_interval);
        alpha[s] = union_measure(buf, m);
    }
    free(buf);
}

/*
 * All listed edges, in increasing id order.  An edge is listed when
 * 0 < alpha < 1 (its coefficient differs from both pure media) or when its
 * endpoints lie in different media (it carries a polarisation flux).
 * Returns the number of listed edges; arrays are filled up to cap entries.
 * Per atom, every edge that can meet its ball receives that ball's interval;
 * the intervals are then sorted by (edge, t0, t1) and merged edge by edge.
 */
long orc_crossing_edges(const int n[3], const double o[3], double h,
                        const double *atoms, long na, const uint8_t *inside,
                        long cap, int64_t *ids, double *alpha, double *rp,
                        int8_t *sign)
{
    long N = (long)n[0] * n[1] * n[2];
    long nint = 0, capint = 1024;
    interval *iv = (interval *)malloc(sizeof(interval) * (size_t)capint);
    for (long q = 0; q < na; ++q) {
        const double *p = atoms + 5 * q;
        long lo[3], hi[3];
        for (int d = 0; d < 3; ++d) node_range(n, o, h, d, p[d], p[3] + h, &lo[d], &hi[d]);
        for (int d = 0; d < 3; ++d) {
            long stride_lim = n[d] - 1;
            for (long k = lo[2]; k <= hi[2]; ++k)
                for (long j = lo[1]; j <= hi[1]; ++j)
                    for (long i = lo[0]; i <= hi[0]; ++i) {
                        long c = (d == 0) ? i : ((d == 1) ? j : k);
                        if (c >= stride_lim) continue;
                        double xa[3] = {coord(o, h, 0, i), coord(o, h, 1, j), coord(o, h, 2, k)};
                        double t0, t1;
                        if (!ball_interval(xa, d, h, p, &t0, &t1)) continue;
                        if (nint == capint) {
                            capint *= 2;
                            iv = (interval *)realloc(iv, sizeof(interval) * (size_t)capint);
                        }
                        iv[nint].id = (int64_t)d * N + (k * n[1] + j) * n[0] + i;
                        iv[nint].t0 = t0;
                        iv[nint].t1 = t1;
                        ++nint;
                    }
        }
    }
    qsort(iv, (size_t)nint, sizeof(interval), cmp_interval);

    long count = 0, g = 0;
    for (int d = 0; d < 3; ++d) {
        long stride = (d == 0) ? 1 : ((d == 1) ? n[0] : (long)n[0] * n[1]);
        for (long a = 0; a < N; ++a) {
            long i = a % n[0], j = (a / n[0]) % n[1], k = a / ((long)n[0] * n[1]);
            long c = (d == 0) ? i : ((d == 1) ? j : k);
            if (c >= n[d] - 1) continue;
            int64_t id = (int64_t)d * N + a;
            while (g < nint && iv[g].id < id) ++g;
            long g1 = g;
            while (g1 < nint && iv[g1].id == id) ++g1;
            double al = union_measure(iv + g, g1 - g);
            g = g1;
            int ina = inside[a], inb = inside[a + stride];
            if ((al > 0.0 && al < 1.0) || ina != inb) {
                if (count < cap) {
                    int sg;
                    ids[count] = id;
                    alpha[count] = al;
                    edge_point(n, o, h, id, al, ina, inb, rp + 3 * count, &sg);
                    sign[count] = (int8_t)sg;
                }
                ++count;
            }
        }
    }
    free(iv);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Coefficients (Sec. 3.1 trapezoidal/vertex quadrature, Sec. 3.2 WHA).      */
/* ------------------------------------------------------------------------ */
static double wha(double alpha, double eps_in, double eps_out)
{
    return 1.0 / (alpha / eps_in + (1.0 - alpha) / eps_out);
}

void orc_assemble(const int n[3], double h, const uint8_t *inside, long ncross,
                  const int64_t *ids, const double *alpha, double eps_in,
                  double eps_out, double kD, double *Wx, double *Wy, double *Wz,
                  double *kap, double *diag)
{
    long N = (long)n[0] * n[1] * n[2];
    double *W[3] = {Wx, Wy, Wz};
    long stride[3] = {1, n[0], (long)n[0] * n[1]};
    double kap_s = eps_out * kD * kD * h * h * h;
    for (long a = 0; a < N; ++a) {
        long ijk[3] = {a % n[0], (a / n[0]) % n[1], a / ((long)n[0] * n[1])};
        for (int d = 0; d < 3; ++d)
            W[d][a] = (ijk[d] < n[d] - 1) ? (inside[a] ? eps_in : eps_out) * h : 0.0;
        kap[a] = inside[a] ? 0.0 : kap_s;
    }
    for (long s = 0; s < ncross; ++s) {
        int d = (int)(ids[s] / N);
        long a = ids[s] % N;
        W[d][a] = wha(alpha[s], eps_in, eps_out) * h;
    }
    for (long a = 0; a < N; ++a) {
        long ijk[3] = {a % n[0], (a / n[0]) % n[1], a / ((long)n[0] * n[1])};
        int interior = 1;
        for (int d = 0; d < 3; ++d)
            if (ijk[d] == 0 || ijk[d] == n[d] - 1) interior = 0;
        if (!interior) {
            diag[a] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            s = s + W[d][a - stride[d]];
            s = s + W[d][a];
        }
        diag[a] = s + kap[a];
    }
}

static int is_boundary(const int *n, long a)
{
    long i = a % n[0], j = (a / n[0]) % n[1], k = a / ((long)n[0] * n[1]);
    return i == 0 || j == 0 || k == 0 || i == n[0] - 1 || j == n[1] - 1 || k == n[2] - 1;
}

/* Dirichlet values on the box faces (Sec. 2.3): zero, or the screened
 * Coulomb sum phi = (l_B / eps_s) sum_i q_i exp(-k r) / r (k = 0 gives the
 * Coulomb condition, k = k_D the Debye-Hueckel one). */
void orc_bc_values(const int n[3], const double o[3], double h,
                   const double *atoms, long na, double lB, double eps_out,
                   double k, double *phib)
{
    long N = (long)n[0] * n[1] * n[2];
    for (long a = 0; a < N; ++a) {
        if (!is_boundary(n, a)) {
            phib[a] = 0.0;
            continue;
        }
        double x[3];
        node_pos(n, o, h, a, x);
        double s = 0.0;
        for (long q = 0; q < na; ++q) {
            const double *p = atoms + 5 * q;
            double dx = x[0] - p[0], dy = x[1] - p[1], dz = x[2] - p[2];
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            s += p[4] * exp(-k * r) / r;
        }
        phib[a] = (lB / eps_out) * s;
    }
}

/* Right-hand side R(v) = int rho^f v of Eq. RVop with trilinear v, scaled
 * by 4 pi l_B, plus the couplings of interior nodes to Dirichlet nodes.
 * Returns -1 if a charge's cell touches the boundary, else 0. */
int orc_rhs(const int n[3], const double o[3], double h, const double *atoms,
            long na, double lB, const double *Wx, const double *Wy,
            const double *Wz, const double *phib, double *f)
{
    long N = (long)n[0] * n[1] * n[2];
    long stride[3] = {1, n[0], (long)n[0] * n[1]};
    const double *W[3] = {Wx, Wy, Wz};
    memset(f, 0, sizeof(double) * (size_t)N);
    for (long q = 0; q < na; ++q) {
        const double *p = atoms + 5 * q;
        long c[3];
        double w[3][2];
        for (int d = 0; d < 3; ++d) {
            double u = (p[d] - o[d]) / h;
            c[d] = clampl((long)floor(u), 0, n[d] - 2);
            double t = u - (double)c[d];
            w[d][0] = 1.0 - t;
            w[d][1] = t;
            if (c[d] < 1 || c[d] + 1 > n[d] - 2) return -1;
        }
        double coef = 4.0 * M_PI * lB * p[4];
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    long a = ((c[2] + dk) * n[1] + (c[1] + dj)) * n[0] + (c[0] + di);
                    f[a] += coef * (w[0][di] * w[1][dj] * w[2][dk]);
                }
    }
    for (long a = 0; a < N; ++a) {
        if (is_boundary(n, a)) continue;
        for (int d = 0; d < 3; ++d) {
            long m = a - stride[d], pl = a + stride[d];
            if (is_boundary(n, m)) f[a] += W[d][m] * phib[m];
            if (is_boundary(n, pl)) f[a] += W[d][a] * phib[pl];
        }
    }
    return 0;
}

/* y = A x on interior nodes (A = G^T W G + C restricted to interior
 * unknowns; boundary entries of x are treated as zero, y is zero there). */
void orc_apply(const int n[3], const double *Wx, const double *Wy,
               const double *Wz, const double *diag, const double *x, double *y)
{
    long N = (long)n[0] * n[1] * n[2];
    long sy = n[0], sz = (long)n[0] * n[1];
    memset(y, 0, sizeof(double) * (size_t)N);
    for (long k = 1; k < n[2] - 1; ++k)
        for (long j = 1; j < n[1] - 1; ++j)
            for (long i = 1; i < n[0] - 1; ++i) {
                long a = k * sz + j * sy + i;
                double s = 0.0;
                if (i > 1) s += Wx[a - 1] * x[a - 1];
                if (i < n[0] - 2) s += Wx[a] * x[a + 1];
                if (j > 1) s += Wy[a - sy] * x[a - sy];
                if (j < n[1] - 2) s += Wy[a] * x[a + sy];
                if (k > 1) s += Wz[a - sz] * x[a - sz];
                if (k < n[2] - 2) s += Wz[a] * x[a + sz];
                y[a] = diag[a] * x[a] - s;
            }
}

static double dot_interior(const int *n, const double *u, const double *v)
{
    long sy = n[0], sz = (long)n[0] * n[1];
    double s = 0.0;
    for (long k = 1; k < n[2] - 1; ++k)
        for (long j = 1; j < n[1] - 1; ++j)
            for (long i = 1; i < n[0] - 1; ++i) {
                long a = k * sz + j * sy + i;
                s += u[a] * v[a];
            }
    return s;
}

/*
 * Jacobi-preconditioned conjugate gradient on the interior unknowns
 * (the Krylov solve of Eq. matrixequation; the paper uses CG, Sec. 4).
 * Zero initial guess.  Stops when ||f - A x||_2 <= rtol ||f||_2, checking the
 * true residual whenever the recursive one passes the test.
 * Returns 0 on convergence, 1 on reaching max_iter.
 */
int orc_pcg(const int n[3], const double *Wx, const double *Wy, const double *Wz,
            const double *diag, const double *f, double rtol, long max_iter,
            double *x, long *iters, double *relres)
{
    long N = (long)n[0] * n[1] * n[2];
    double *r = (double *)calloc((size_t)N, sizeof(double));
    double *z = (double *)calloc((size_t)N, sizeof(double));
    double *p = (double *)calloc((size_t)N, sizeof(double));
    double *q = (double *)calloc((size_t)N, sizeof(double));
    uint8_t *in = (uint8_t *)calloc((size_t)N, 1); /* 1 on interior unknowns */
    for (long a = 0; a < N; ++a) in[a] = (uint8_t)!is_boundary(n, a);
    memset(x, 0, sizeof(double) * (size_t)N);
    double fnorm = sqrt(dot_interior(n, f, f));
    int status = 1;
    long it = 0;
    double rel = 0.0;
    if (fnorm == 0.0) {
        status = 0;
        goto done;
    }
    for (long a = 0; a < N; ++a) r[a] = in[a] ? f[a] : 0.0;
    for (;;) {
        /* (re)start from the current residual r */
        for (long a = 0; a < N; ++a) z[a] = in[a] ? r[a] / diag[a] : 0.0;
        memcpy(p, z, sizeof(double) * (size_t)N);
        double rho = dot_interior(n, r, z);
        int restart = 0;
        while (it < max_iter) {
            orc_apply(n, Wx, Wy, Wz, diag, p, q);
            double sigma = dot_interior(n, p, q);
            double al = rho / sigma;
            for (long a = 0; a < N; ++a) {
                if (!in[a]) continue;
                x[a] += al * p[a];
                r[a] -= al * q[a];
            }
            ++it;
            double rn = sqrt(dot_interior(n, r, r));
            if (rn <= rtol * fnorm) {
                orc_apply(n, Wx, Wy, Wz, diag, x, q);
                for (long a = 0; a < N; ++a) r[a] = in[a] ? f[a] - q[a] : 0.0;
                rel = sqrt(dot_interior(n, r, r)) / fnorm;
                if (rel <= rtol) {
                    status = 0;
                    goto done;
                }
                restart = 1;
                break;
            }
            for (long a = 0; a < N; ++a) z[a] = in[a] ? r[a] / diag[a] : 0.0;
            double rho1 = dot_interior(n, r, z);
            double be = rho1 / rho;
            rho = rho1;
            for (long a = 0; a < N; ++a) p[a] = z[a] + be * p[a];
        }
        if (!restart) break;
    }
    orc_apply(n, Wx, Wy, Wz, diag, x, q);
    for (long a = 0; a < N; ++a) r[a] = in[a] ? f[a] - q[a] : 0.0;
    rel = sqrt(dot_interior(n, r, r)) / fnorm;
done:
    *iters = it;
    *relres = rel;
    free(r);
    free(z);
    free(p);
    free(q);
    free(in);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Analytic N-body terms (Sec. 3.3).                                          */
/* ------------------------------------------------------------------------ */

/* Phi_t = sum_i q_i exp(-k r_ti) / r_ti at each target t. */
void orc_coulomb_phi(const double *tgt, long nt, const double *atoms, long na,
                     double k, double *out)
{
    for (long t = 0; t < nt; ++t) {
        double s = 0.0;
        for (long q = 0; q < na; ++q) {
            const double *p = atoms + 5 * q;
            double dx = tgt[3 * t] - p[0], dy = tgt[3 * t + 1] - p[1], dz = tgt[3 * t + 2] - p[2];
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            s += p[4] * exp(-k * r) / r;
        }
        out[t] = s;
    }
}

/* Psi_t = sum_i q_i (r_t - r_i) . n_t / |r_t - r_i|^3 with n_t = sign_t e_{dir_t}. */
void orc_coulomb_psi(const double *tgt, const int8_t *dir, const int8_t *sign,
                     long nt, const double *atoms, long na, double *out)
{
    for (long t = 0; t < nt; ++t) {
        double s = 0.0;
        for (long q = 0; q < na; ++q) {
            const double *p = atoms + 5 * q;
            double u[3] = {tgt[3 * t] - p[0], tgt[3 * t + 1] - p[1], tgt[3 * t + 2] - p[2]};
            double r2 = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
            double r = sqrt(r2);
            s += p[4] * ((double)sign[t] * u[dir[t]]) / (r2 * r);
        }
        out[t] = s;
    }
}

/* E_coul = (l_B / eps_m) sum_{i<j} q_i q_j / r_ij   (Sec. 3.3). */
double orc_ecoul(const double *atoms, long na, double lB, double eps_in)
{
    double s = 0.0;
    for (long i = 0; i < na; ++i)
        for (long j = 0; j < i; ++j) {
            const double *a = atoms + 5 * i, *b = atoms + 5 * j;
            double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
            s += a[4] * b[4] / sqrt((dx * dx + dy * dy) + dz * dz);
        }
    return (lB / eps_in) * s;
}

/*
 * Energy terms from the solved potential phi (full grid, boundary values
 * included).  For each flux edge (endpoints in different media):
 *   F_e = W_e (phi_in - phi_out)   outward flux of D^eff through the dual
 *                                   face, Eq. Dnvh_approx (times 4 pi l_B)
 *   q_p = (1/eps_s - 1/eps_m) F_e / (4 pi l_B)   placed at r_p (Sec. 3.3.1)
 *   E_pol      = 1/2 (1/eps_s - 1/eps_m) sum_e F_e Phi_e / (4 pi)
 *   E_ion_flux = -1/2 (1/eps_s) sum_e F_e Phi_e / (4 pi)   (second integral
 *                of Eq. energy_ion)
 *   E_ion_surf = 1/2 sum_e phi(r_p) h^2 Psi_e / (4 pi)     (first integral of
 *                Eq. energy_ion on the staircase faces, phi(r_p) from Eq. phi0)
 * out = {e_coul, e_pol, e_ion_surf, e_ion_flux, e_total, sum_F/(4 pi l_B)}.
 */
void orc_energy(const int n[3], const double o[3], double h, const uint8_t *inside,
                long ncross, const int64_t *ids, const double *alpha,
                const double *rp, const int8_t *sign, const double *Wx,
                const double *Wy, const double *Wz, const double *phi,
                const double *atoms, long na, double lB, double eps_in,
                double eps_out, double *out)
{
    const double *W[3] = {Wx, Wy, Wz};
    double S = 0.0, I = 0.0, F = 0.0;
    (void)inside;
    for (long s = 0; s < ncross; ++s) {
        if (sign[s] == 0) continue;
        int d;
        long a, b;
        edge_nodes(n, ids[s], &d, &a, &b);
        long in = sign[s] > 0 ? a : b, out_n = sign[s] > 0 ? b : a;
        double Fe = W[d][a] * (phi[in] - phi[out_n]);
        int8_t dd = (int8_t)d;
        double Phi, Psi;
        orc_coulomb_phi(rp + 3 * s, 1, atoms, na, 0.0, &Phi);
        orc_coulomb_psi(rp + 3 * s, &dd, sign + s, 1, atoms, na, &Psi);
        double al = alpha[s];
        double pin = phi[in], pout = phi[out_n];
        double phip = pin + (al / eps_in) * (pout - pin) / (al / eps_in + (1.0 - al) / eps_out);
        S += Fe * Phi;
        I += phip * (h * h) * Psi;
        F += Fe;
    }
    double e_coul = orc_ecoul(atoms, na, lB, eps_in);
    double e_pol = 0.5 * (1.0 / eps_out - 1.0 / eps_in) * S / (4.0 * M_PI);
    double e_ion_flux = -0.5 * (1.0 / eps_out) * S / (4.0 * M_PI);
    double e_ion_surf = 0.5 * I / (4.0 * M_PI);
    out[0] = e_coul;
    out[1] = e_pol;
    out[2] = e_ion_surf;
    out[3] = e_ion_flux;
    out[4] = e_coul + e_pol + e_ion_surf + e_ion_flux;
    out[5] = F / (4.0 * M_PI * lB);
}

/* Coefficients of selected interior nodes computed from scratch by brute
 * force (6 face weights in the order -x,+x,-y,+y,-z,+z, then kappa h^3 and
 * the diagonal), for sampled checks at sizes the full oracle cannot reach. */
void orc_node_coeffs(const int n[3], const double o[3], double h,
                     const double *atoms, long na, double eps_in,
                     double eps_out, double kD, const int64_t *nodes,
                     long count, double *out)
{
    long N = (long)n[0] * n[1] * n[2];
    long stride[3] = {1, n[0], (long)n[0] * n[1]};
    double kap_s = eps_out * kD * kD * h * h * h;
    for (long s = 0; s < count; ++s) {
        long a = nodes[s];
        double *o8 = out + 8 * s;
        uint8_t ia;
        int64_t aa = a;
        orc_classify_nodes(n, o, h, atoms, na, &aa, 1, &ia);
        double sum = 0.0;
        for (int d = 0; d < 3; ++d) {
            for (int side = 0; side < 2; ++side) {
                long lo = side == 0 ? a - stride[d] : a;
                int64_t id = (int64_t)d * N + lo;
                int64_t lo64 = lo, hi64 = lo + stride[d];
                uint8_t in_lo, in_hi;
                orc_classify_nodes(n, o, h, atoms, na, &lo64, 1, &in_lo);
                orc_classify_nodes(n, o, h, atoms, na, &hi64, 1, &in_hi);
                double al;
                orc_edge_alpha(n, o, h, atoms, na, &id, 1, &al);
                double w;
                if ((al > 0.0 && al < 1.0) || in_lo != in_hi)
                    w = wha(al, eps_in, eps_out) * h;
                else
                    w = (in_lo ? eps_in : eps_out) * h;
                o8[2 * d + side] = w;
            }
        }
        for (int d = 0; d < 3; ++d) {
            sum = sum + o8[2 * d];
            sum = sum + o8[2 * d + 1];
        }
        double kap = ia ? 0.0 : kap_s;
        o8[6] = kap;
        o8[7] = sum + kap;
    }
}

/* ------------------------------------------------------------------------ */
/* First integral of Eq. energy_ion (Sec. 3.3.2) on a re-triangulated       */
/* surface.  The surface is re-triangulated cell by cell by marching cubes  */
/* whose vertices are the analytic intersection points r_p of the crossing  */
/* edges (edges whose end nodes differ in medium), with analytic normals;    */
/* the integral takes the vertex rule T_j/3 on every triangle and phi at the */
/* vertices from Eq. phi0.                                                   */
/*                                                                          */
/* Triangulation of one cell, without a case table: on each of the six      */
/* faces the crossing edges are joined in pairs (two crossings: one         */
/* segment; four, the ambiguous face, two segments that each cut off one    */
/* inside corner, so the two cells sharing a face agree and the surface is  */
/* closed).  Every crossing edge of the cell lies on two faces, so the      */
/* segments form closed loops.  Each loop starts at its lowest cell-edge    */
/* index, goes first to the smaller of that vertex's two neighbours, and is */
/* cut into the fan of triangles (v0, v_m, v_m+1).                           */
/* ------------------------------------------------------------------------ */

/* cell corners: bit 0 = +x, bit 1 = +y, bit 2 = +z.  Cell edges 0..11:
 * along x (0,1) (2,3) (4,5) (6,7); along y (0,2) (1,3) (4,6) (5,7);
 * along z (0,4) (1,5) (2,6) (3,7). */
static const int mc_edge_corner[12][2] = {
    {0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7},
    {0, 4}, {1, 5}, {2, 6}, {3, 7}};
/* faces as four corners in cyclic order */
static const int mc_face[6][4] = {
    {0, 2, 6, 4}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 3, 7, 6}, {0, 1, 3, 2}, {4, 5, 7, 6}};

static int mc_edge_of(int ca, int cb)
{
    for (int e = 0; e < 12; ++e)
        if ((mc_edge_corner[e][0] == ca && mc_edge_corner[e][1] == cb) ||
            (mc_edge_corner[e][0] == cb && mc_edge_corner[e][1] == ca))
            return e;
    return -1;
}

/* index of edge id in the sorted crossing list, -1 if absent */
static long find_edge(const int64_t *ids, long ncross, int64_t id)
{
    long lo = 0, hi = ncross - 1;
    while (lo <= hi) {
        long mid = lo + (hi - lo) / 2;
        if (ids[mid] == id) return mid;
        if (ids[mid] < id) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* Triangles of cell (i,j,k): writes up to 12 triangles as triples of
 * crossing-list indices into tri (fan order) and their areas; returns the
 * triangle count. */
static int mc_cell(const int *n, const uint8_t *inside, long ncross, const int64_t *ids,
                   const double *rp, long i, long j, long k, long *tri, double *area)
{
    long N = (long)n[0] * n[1] * n[2];
    long node[8];
    int ins[8];
    int any_in = 0, any_out = 0;
    for (int c = 0; c < 8; ++c) {
        long a = ((k + ((c >> 2) & 1)) * n[1] + (j + ((c >> 1) & 1))) * n[0] + (i + (c & 1));
        node[c] = a;
        ins[c] = inside[a] ? 1 : 0;
        if (ins[c]) any_in = 1;
        else any_out = 1;
    }
    if (!(any_in && any_out)) return 0;
    long vert[12];
    for (int e = 0; e < 12; ++e) {
        int ca = mc_edge_corner[e][0], cb = mc_edge_corner[e][1];
        vert[e] = -1;
        if (ins[ca] != ins[cb]) {
            int d = e / 4;
            vert[e] = find_edge(ids, ncross, (int64_t)d * N + node[ca]);
        }
    }
    int nbr[12][2], deg[12];
    for (int e = 0; e < 12; ++e) deg[e] = 0;
    for (int f = 0; f < 6; ++f) {
        const int *c = mc_face[f];
        int fe[4];
        for (int q = 0; q < 4; ++q) fe[q] = mc_edge_of(c[q], c[(q + 1) & 3]);
        int cr[4], m = 0;
        for (int q = 0; q < 4; ++q)
            if (ins[c[q]] != ins[c[(q + 1) & 3]]) cr[m++] = q;
        int pairs[2][2], np = 0;
        if (m == 2) {
            pairs[0][0] = fe[cr[0]];
            pairs[0][1] = fe[cr[1]];
            np = 1;
        } else if (m == 4) {
            /* cut off each inside corner: corner q lies between face edges
             * q-1 and q */
            int q0 = ins[c[0]] ? 0 : 1;
            pairs[0][0] = fe[(q0 + 3) & 3];
            pairs[0][1] = fe[q0];
            pairs[1][0] = fe[(q0 + 1) & 3];
            pairs[1][1] = fe[(q0 + 2) & 3];
            np = 2;
        }
        for (int p = 0; p < np; ++p) {
            int a = pairs[p][0], b = pairs[p][1];
            nbr[a][deg[a]++] = b;
            nbr[b][deg[b]++] = a;
        }
    }
    int seen[12] = {0};
    int nt = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
        if (ins[mc_edge_corner[e0][0]] == ins[mc_edge_corner[e0][1]] || seen[e0]) continue;
        int loop[12], len = 0;
        int prev = e0;
        int cur = nbr[e0][0] < nbr[e0][1] ? nbr[e0][0] : nbr[e0][1];
        loop[len++] = e0;
        seen[e0] = 1;
        while (cur != e0 && len < 12) {
            loop[len++] = cur;
            seen[cur] = 1;
            int nx = nbr[cur][0] == prev ? nbr[cur][1] : nbr[cur][0];
            prev = cur;
            cur = nx;
        }
        for (int m = 1; m + 1 < len; ++m) {
            long a = vert[loop[0]], b = vert[loop[m]], c = vert[loop[m + 1]];
            if (a < 0 || b < 0 || c < 0) continue;
            const double *pa = rp + 3 * a, *pb = rp + 3 * b, *pc = rp + 3 * c;
            double u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
            double v[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
            double x = u[1] * v[2] - u[2] * v[1];
            double y = u[2] * v[0] - u[0] * v[2];
            double z = u[0] * v[1] - u[1] * v[0];
            tri[3 * nt] = a;
            tri[3 * nt + 1] = b;
            tri[3 * nt + 2] = c;
            area[nt] = 0.5 * sqrt((x * x + y * y) + z * z);
            ++nt;
        }
    }
    return nt;
}

/* Vertex weights of the re-triangulated surface: W[s] = sum of T_j / 3 over
 * the triangles that have crossing point s as a vertex (0 for edges whose
 * end nodes lie in the same medium).  Cells are visited in node order. */
void orc_mc_weights(const int n[3], const uint8_t *inside, long ncross, const int64_t *ids,
                    const double *rp, double *W)
{
    long tri[36];
    double area[12];
    for (long s = 0; s < ncross; ++s) W[s] = 0.0;
    for (long k = 0; k + 1 < n[2]; ++k)
        for (long j = 0; j + 1 < n[1]; ++j)
            for (long i = 0; i + 1 < n[0]; ++i) {
                int nt = mc_cell(n, inside, ncross, ids, rp, i, j, k, tri, area);
                for (int t = 0; t < nt; ++t)
                    for (int v = 0; v < 3; ++v) W[tri[3 * t + v]] += area[t] / 3.0;
            }
}

/* Analytic outward normal of the union of balls at each crossing point with
 * sign != 0: the unit vector from the centre of the ball whose sphere passes
 * closest to the point (smallest | |r_p - c_i| - R_i |, ties to the lower
 * atom index).  Zero for the other edges. */
void orc_mc_normals(long ncross, const double *rp, const int8_t *sign, const double *atoms,
                    long na, double *nrm)
{
    for (long s = 0; s < ncross; ++s) {
        double *o = nrm + 3 * s;
        o[0] = o[1] = o[2] = 0.0;
        if (sign[s] == 0) continue;
        const double *p = rp + 3 * s;
        long best = -1;
        double bdev = 0.0, bd = 0.0;
        for (long a = 0; a < na; ++a) {
            const double *c = atoms + 5 * a;
            double dx = p[0] - c[0], dy = p[1] - c[1], dz = p[2] - c[2];
            double d = sqrt((dx * dx + dy * dy) + dz * dz);
            double dev = fabs(d - c[3]);
            if (best < 0 || dev < bdev) {
                best = a;
                bdev = dev;
                bd = d;
            }
        }
        const double *c = atoms + 5 * best;
        o[0] = (p[0] - c[0]) / bd;
        o[1] = (p[1] - c[1]) / bd;
        o[2] = (p[2] - c[2]) / bd;
    }
}

/* Psi with a general normal: sum_i q_i (r_t - r_i).n_t / |r_t - r_i|^3 */
void orc_coulomb_psi_n(const double *tgt, const double *nrm, long nt, const double *atoms,
                       long na, double *out)
{
    for (long t = 0; t < nt; ++t) {
        const double *p = tgt + 3 * t, *nv = nrm + 3 * t;
        double acc = 0.0;
        for (long a = 0; a < na; ++a) {
            const double *c = atoms + 5 * a;
            double dx = p[0] - c[0], dy = p[1] - c[1], dz = p[2] - c[2];
            double r2 = (dx * dx + dy * dy) + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            acc += c[4] * ((dx * nv[0] + dy * nv[1]) + dz * nv[2]) / (r2 * r);
        }
        out[t] = acc;
    }
}

/* E_ion first integral on the re-triangulated surface:
 * 1/2 sum_s W_s phi(r_s) Psi_n(r_s) / (4 pi), phi(r_s) by Eq. phi0 from the
 * edge's two end nodes (alpha = inside fraction from the inside node). */
double orc_energy_ion_mc(const int n[3], long ncross, const int64_t *ids, const double *alpha,
                         const double *rp, const int8_t *sign, const double *W,
                         const double *nrm, const double *phi, const double *atoms, long na,
                         double eps_in, double eps_out)
{
    double I = 0.0;
    for (long s = 0; s < ncross; ++s) {
        if (sign[s] == 0 || W[s] == 0.0) continue;
        int d;
        long a, b;
        edge_nodes(n, ids[s], &d, &a, &b);
        long in = sign[s] > 0 ? a : b, out_n = sign[s] > 0 ? b : a;
        double al = alpha[s];
        double pin = phi[in], pout = phi[out_n];
        double phip = pin + (al / eps_in) * (pout - pin) / (al / eps_in + (1.0 - al) / eps_out);
        double psi;
        orc_coulomb_psi_n(rp + 3 * s, nrm + 3 * s, 1, atoms, na, &psi);
        I += W[s] * phip * psi;
    }
    return 0.5 * I / (4.0 * M_PI);
}
