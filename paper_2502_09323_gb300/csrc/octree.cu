// Octree brick grid of the linear PB hot path.
//
// The paper refines its Cartesian grid as an octree near the molecular
// surface (Sec. 3, Sec. 3.4) and leaves the treatment of hanging nodes to
// prior work.  This file implements the following reading:
//
//  * Domain: n0^3 coarse bricks of side 8 h_bulk, centred on the bounding
//    box of the atom spheres (n0 = ceil(fill * extent / (8 h_bulk))), or an
//    explicit origin and n0.  Levels l = 0..Lmax with cell size
//    h_l = h_bulk / 2^l, h_Lmax = h_fine.  Positions are integers in units
//    of h_fine ("node units"); node-unit position P sits at origin + P*h_fine.
//  * A level-l brick (8^3 cells) is split when its closed box lies within
//    refine_dist of some atom's sphere surface (dmin <= R + d and
//    dmax >= R - d, compared as squares); then leaves touching across a
//    face, an edge or a corner are split until their levels differ by at
//    most one (2:1 balance).  Leaves are ordered by the Morton code of their
//    low corner; brick b owns the 8^3 low-corner nodes of its cells.
//  * Nodes: boundary (a coordinate is 0 or the domain side), hanging (a
//    touching leaf does not have the node on its lattice; its value is the
//    mean of the 2 or 4 coarse corners of the edge or face it lies on),
//    regular otherwise.
//  * Operator (Eq. matrixequation in element form): every leaf cell of size
//    h adds (eps_e h / 4)(d_a - d_b)(d_a - d_b)^T for each of its 12 edges
//    (eps_e of Eq. WHA) and eps_s k_D^2 h^3 / 8 at each solvent corner;
//    A = P^T K P on the regular interior nodes, P the hanging-node
//    interpolation.  A node whose 8 cells share its level and whose 6
//    neighbours are regular and owned at that level has the uniform 7-point
//    row (W_e = eps_e h, C = kappa h^3): a "pure" row, applied as a brick
//    stencil with the compressed operator.  The other regular rows (next to
//    a level change) are assembled once as explicit CSR rows.
//  * refine_dist >= max(R_max, h_fine, 1.5 h_bulk): every solute node, edge
//    meeting the surface and charge cell then lies in the all-finest region
//    (where the octree equals the uniform grid at h_fine), and every
//    level-transition row sees solvent only.
//
// The edges meeting the surface are found by the uniform-grid pass run on
// the finest lattice of the domain (the same alpha, r_p and signs as a
// uniform grid at h_fine), then renumbered by slot.

#include <math.h>

#include <algorithm>
#include <chrono>
#include <cub/cub.cuh>
#include <vector>

#include "pb_internal.h"

namespace pbg {
namespace {

constexpr int OT = 256;       // threads of the element-wise octree kernels
constexpr int OB = 256;       // threads of the brick kernels (2 nodes each)
constexpr int MAXE = 160;     // distinct columns of one level-transition row
constexpr int MAXA = 48;      // rows of P^T that reach one transition row

enum : uint32_t {
    OERR_SOLUTE_TRANSITION = 1u,  // a level-transition row touched a solute node
    OERR_ROW_OVERFLOW = 2u,       // a transition row has too many columns
    OERR_CROSS_OWNER = 4u,        // a listed edge outside the all-finest region
    OERR_HANGING_PARENT = 8u,     // a hanging node's parent is not regular/boundary
    OERR_DEPOSIT = 16u,           // a charge cell corner is not a regular finest node
};

struct MinOpD {
    __device__ double operator()(double a, double b) const { return a < b ? a : b; }
};
struct MaxOpD {
    __device__ double operator()(double a, double b) const { return a > b ? a : b; }
};
struct OrOpU {
    __device__ unsigned operator()(unsigned a, unsigned b) const { return a | b; }
};

__host__ __device__ __forceinline__ int spc(int Lmax, int level) { return 1 << (Lmax - level); }

__device__ __forceinline__ long long cidx(const OctDev &t, int cx, int cy, int cz) {
    return ((long long)cz * t.nf + cy) * t.nf + cx;
}

// world coordinate of a node-unit position (one multiply, one add)
__device__ __forceinline__ double wpos(const OctDev &t, int d, int P) {
    return __dadd_rn(t.o[d], __dmul_rn((double)P, t.hf));
}

// largest and smallest lattice spacing among the leaves whose closed box
// holds P
__device__ int touch_spacings(const OctDev &t, int px, int py, int pz, int &smin) {
    const int P[3] = {px, py, pz};
    int smax = 0;
    smin = 1 << 30;
    for (int o = 0; o < 8; ++o) {
        int c[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            const int off = (o >> d) & 1;
            if (off && (P[d] & 7) != 0) {
                ok = false;  // same cell as off = 0
                break;
            }
            c[d] = (P[d] >> 3) - off;
            if (c[d] < 0 || c[d] >= t.nf) ok = false;
        }
        if (!ok) continue;
        const int s = spc(t.Lmax, t.lev[cidx(t, c[0], c[1], c[2])]);
        smax = max(smax, s);
        smin = min(smin, s);
    }
    return smax;
}

__device__ __forceinline__ int touch_smax(const OctDev &t, int px, int py, int pz) {
    int smin;
    return touch_spacings(t, px, py, pz, smin);
}

// 0 regular interior, 1 boundary, 2 hanging
__device__ int pos_kind(const OctDev &t, int px, int py, int pz) {
    if (px == 0 || py == 0 || pz == 0 || px == t.NL || py == t.NL || pz == t.NL) return 1;
    const int s = touch_smax(t, px, py, pz);
    if ((px % s) || (py % s) || (pz % s)) return 2;
    return 0;
}

// slot owning position P (all coordinates < NL), or -1 if P is not on the
// lattice of the leaf that contains it
__device__ long long owner_slot(const OctDev &t, int px, int py, int pz) {
    if (px < 0 || py < 0 || pz < 0 || px >= t.NL || py >= t.NL || pz >= t.NL) return -1;
    const int b = t.bmap[cidx(t, px >> 3, py >> 3, pz >> 3)];
    const int4 L = t.blow[b];
    const int s = spc(t.Lmax, L.w);
    const int dx = px - L.x, dy = py - L.y, dz = pz - L.z;
    if ((dx % s) || (dy % s) || (dz % s)) return -1;
    return ((long long)b << 9) + ((dz / s) * 8 + dy / s) * 8 + dx / s;
}

__device__ __forceinline__ void slot_pos(const OctDev &t, long long a, int P[3], int &level) {
    const int4 L = t.blow[a >> 9];
    const int loc = (int)(a & 511);
    const int s = spc(t.Lmax, L.w);
    P[0] = L.x + s * (loc & 7);
    P[1] = L.y + s * ((loc >> 3) & 7);
    P[2] = L.z + s * (loc >> 6);
    level = L.w;
}

// parents of hanging position P: 2 (edge) or 4 (face) coarse corners
__device__ int hang_parents(const OctDev &t, const int P[3], int par[4][3], double &w) {
    const int s = touch_smax(t, P[0], P[1], P[2]);
    const int half = s >> 1;
    int dims[3], nd = 0;
    for (int d = 0; d < 3; ++d)
        if (P[d] % s) dims[nd++] = d;
    const int np = 1 << nd;
    for (int q = 0; q < np; ++q) {
        for (int d = 0; d < 3; ++d) par[q][d] = P[d];
        for (int e = 0; e < nd; ++e) par[q][dims[e]] += ((q >> e) & 1) ? half : -half;
    }
    w = 1.0 / (double)np;
    return np;
}

// Dirichlet value (Sec. 2.3) at a node-unit position: the screened Coulomb
// sum over all atoms in index order (FP64)
struct BcDesc {
    const double *atoms;
    long long na;
    double scale, k;
    int kind;  // PB_BC_*
};

__device__ double bc_at(const OctDev &t, const BcDesc &bd, const int P[3]) {
    if (bd.kind == PB_BC_ZERO) return 0.0;
    const double x = wpos(t, 0, P[0]), y = wpos(t, 1, P[1]), z = wpos(t, 2, P[2]);
    const double *X = bd.atoms, *Y = bd.atoms + bd.na, *Z = bd.atoms + 2 * bd.na,
                 *Q = bd.atoms + 4 * bd.na;
    double acc = 0.0;
    for (long long i = 0; i < bd.na; ++i) {
        const double dx = x - X[i], dy = y - Y[i], dz = z - Z[i];
        const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz)));
        acc += (bd.k > 0.0 ? Q[i] * exp(-bd.k * r) : Q[i]) / r;
    }
    return bd.scale * acc;
}

// ============================================================== build ===
__global__ void __launch_bounds__(OT) k_oct_bbox(const double *__restrict__ atoms, long long na,
                                                 BuildInfo *info) {
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *R = atoms + 3 * na,
                 *Q = atoms + 4 * na;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double rmax = 0.0;
    unsigned err = 0;
    for (long long i = threadIdx.x; i < na; i += OT) {
        const double c[3] = {X[i], Y[i], Z[i]};
        const double r = R[i];
        if (!isfinite(c[0]) || !isfinite(c[1]) || !isfinite(c[2]) || !isfinite(Q[i]) ||
            !isfinite(r) || !(r > 0.0))
            err |= ERRF_ATOM_VALUE;
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], c[d] - r);
            hi[d] = fmax(hi[d], c[d] + r);
        }
        rmax = fmax(rmax, r);
    }
    using BR = cub::BlockReduce<double, OT>;
    using BRU = cub::BlockReduce<unsigned, OT>;
    __shared__ typename BR::TempStorage tmp;
    __shared__ typename BRU::TempStorage tmpu;
    for (int d = 0; d < 3; ++d) {
        double v = BR(tmp).Reduce(lo[d], MinOpD());
        __syncthreads();
        if (threadIdx.x == 0) info->lo[d] = v;
        v = BR(tmp).Reduce(hi[d], MaxOpD());
        __syncthreads();
        if (threadIdx.x == 0) info->hi[d] = v;
    }
    double rm = BR(tmp).Reduce(rmax, MaxOpD());
    unsigned e = BRU(tmpu).Reduce(err, OrOpU());
    if (threadIdx.x == 0) {
        info->rmax = rm;
        info->err = e;
    }
}

// near flag of every level-l box (children of boxes that are not near are
// not near either).  Only an atom whose centre lies within reach = R_max +
// dist of the box can pass the test, so the box scans the atom cell list
// over the cells that meet the box grown by reach (one cell of margin on
// each side); the flag is an OR over atoms, so the order does not matter.
// On a de-refined domain the boxes of the levels coarser than h_tight that
// meet the tight box [tlo, thi] are near too.
__global__ void k_oct_near(const double *__restrict__ atoms, long long na, OctDev t, int level,
                           double dist, double reach, CellList cl,
                           const uint8_t *__restrict__ parent_near, uint8_t *__restrict__ near,
                           bool tight, double3 tlo, double3 thi) {
    const int nl = t.n0 << level;
    const long long nbox = (long long)nl * nl * nl;
    const long long q = blockIdx.x * (long long)OT + threadIdx.x;
    if (q >= nbox) return;
    const int bx = (int)(q % nl), by = (int)((q / nl) % nl), bz = (int)(q / ((long long)nl * nl));
    if (level > 0) {
        const int pl = nl >> 1;
        if (!parent_near[((long long)(bz >> 1) * pl + (by >> 1)) * pl + (bx >> 1)]) {
            near[q] = 0;
            return;
        }
    }
    const int side = 8 * spc(t.Lmax, level);
    const int lo[3] = {bx * side, by * side, bz * side};
    double a[3], b[3];
    for (int d = 0; d < 3; ++d) {
        a[d] = wpos(t, d, lo[d]);
        b[d] = wpos(t, d, lo[d] + side);
    }
    if (tight && a[0] <= thi.x && b[0] >= tlo.x && a[1] <= thi.y && b[1] >= tlo.y &&
        a[2] <= thi.z && b[2] >= tlo.z) {
        near[q] = 1;
        return;
    }
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *R = atoms + 3 * na;
    int c0[3], c1[3];
    bool empty = false;
    for (int d = 0; d < 3; ++d) {
        double u0 = floor((a[d] - reach - cl.lo[d]) / cl.cs) - 1.0;
        double u1 = floor((b[d] + reach - cl.lo[d]) / cl.cs) + 1.0;
        u0 = fmax(u0, 0.0);
        u1 = fmin(u1, (double)cl.dim[d] - 1.0);
        if (!(u0 <= u1)) empty = true;
        c0[d] = empty ? 0 : (int)u0;
        c1[d] = empty ? -1 : (int)u1;
    }
    uint8_t hit = 0;
    for (int cz = c0[2]; cz <= c1[2] && !hit && !empty; ++cz)
    for (int cy = c0[1]; cy <= c1[1] && !hit; ++cy)
    for (int cx = c0[0]; cx <= c1[0] && !hit; ++cx) {
    const int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
    for (int sidx = cl.start[cid]; sidx < cl.start[cid + 1] && !hit; ++sidx) {
        const int i = cl.atom[sidx];
        const double c[3] = {X[i], Y[i], Z[i]};
        double tt[3], u[3];
        for (int d = 0; d < 3; ++d) {
            tt[d] = fmax(fmax(a[d] - c[d], 0.0), c[d] - b[d]);
            u[d] = fmax(fabs(c[d] - a[d]), fabs(c[d] - b[d]));
        }
        const double dmin2 = __dadd_rn(__dadd_rn(__dmul_rn(tt[0], tt[0]), __dmul_rn(tt[1], tt[1])),
                                       __dmul_rn(tt[2], tt[2]));
        const double dmax2 = __dadd_rn(__dadd_rn(__dmul_rn(u[0], u[0]), __dmul_rn(u[1], u[1])),
                                       __dmul_rn(u[2], u[2]));
        const double rin = __dmul_rn(R[i] + dist, R[i] + dist);
        const double ro = R[i] - dist;
        if (dmin2 <= rin && (ro <= 0.0 || dmax2 >= __dmul_rn(ro, ro))) hit = 1;
    }
    }
    near[q] = hit;
}

struct LevelPtrs {
    const uint8_t *p[8];
};

// leaf level from the refinement test: count of consecutive near ancestors
__global__ void k_oct_levels(OctDev t, LevelPtrs near, uint8_t *__restrict__ lev) {
    const long long nc = (long long)t.nf * t.nf * t.nf;
    const long long c = blockIdx.x * (long long)OT + threadIdx.x;
    if (c >= nc) return;
    const int cx = (int)(c % t.nf), cy = (int)((c / t.nf) % t.nf), cz = (int)(c / ((long long)t.nf * t.nf));
    int l = 0;
    while (l < t.Lmax) {
        const int sh = t.Lmax - l, nl = t.n0 << l;
        if (!near.p[l][((long long)(cz >> sh) * nl + (cy >> sh)) * nl + (cx >> sh)]) break;
        ++l;
    }
    lev[c] = (uint8_t)l;
}

// balance step 1: the level each cell needs from its 26 neighbours
__global__ void k_oct_req(OctDev t, const uint8_t *__restrict__ lev, uint8_t *__restrict__ req) {
    const long long nc = (long long)t.nf * t.nf * t.nf;
    const long long c = blockIdx.x * (long long)OT + threadIdx.x;
    if (c >= nc) return;
    const int cx = (int)(c % t.nf), cy = (int)((c / t.nf) % t.nf), cz = (int)(c / ((long long)t.nf * t.nf));
    int r = lev[c];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = cx + dx, y = cy + dy, z = cz + dz;
                if (x < 0 || y < 0 || z < 0 || x >= t.nf || y >= t.nf || z >= t.nf) continue;
                r = max(r, (int)lev[cidx(t, x, y, z)] - 1);
            }
    req[c] = (uint8_t)r;
}

// balance step 2: a level-l box splits if a cell in it needs more than l
__global__ void k_oct_split(OctDev t, int level, const uint8_t *__restrict__ req,
                            uint8_t *__restrict__ split) {
    const int nl = t.n0 << level, f = spc(t.Lmax, level);
    const long long nbox = (long long)nl * nl * nl;
    const long long q = blockIdx.x * (long long)OT + threadIdx.x;
    if (q >= nbox) return;
    const int bx = (int)(q % nl), by = (int)((q / nl) % nl), bz = (int)(q / ((long long)nl * nl));
    uint8_t sp = 0;
    for (int z = 0; z < f && !sp; ++z)
        for (int y = 0; y < f && !sp; ++y)
            for (int x = 0; x < f; ++x)
                if (req[cidx(t, bx * f + x, by * f + y, bz * f + z)] > level) {
                    sp = 1;
                    break;
                }
    split[q] = sp;
}

// balance step 3: new leaf level = the first level whose box does not split
__global__ void k_oct_relevel(OctDev t, LevelPtrs split, uint8_t *__restrict__ lev,
                              int *__restrict__ changed) {
    const long long nc = (long long)t.nf * t.nf * t.nf;
    const long long c = blockIdx.x * (long long)OT + threadIdx.x;
    if (c >= nc) return;
    const int cx = (int)(c % t.nf), cy = (int)((c / t.nf) % t.nf), cz = (int)(c / ((long long)t.nf * t.nf));
    int l = 0;
    while (l < t.Lmax) {
        const int sh = t.Lmax - l, nl = t.n0 << l;
        if (!split.p[l][((long long)(cz >> sh) * nl + (cy >> sh)) * nl + (cx >> sh)]) break;
        ++l;
    }
    if (l != lev[c]) {
        lev[c] = (uint8_t)l;
        *changed = 1;
    }
}

__device__ __forceinline__ unsigned long long morton3(unsigned x, unsigned y, unsigned z) {
    unsigned long long m = 0;
    for (int b = 0; b < 20; ++b) {
        m |= (unsigned long long)((x >> b) & 1u) << (3 * b);
        m |= (unsigned long long)((y >> b) & 1u) << (3 * b + 1);
        m |= (unsigned long long)((z >> b) & 1u) << (3 * b + 2);
    }
    return m;
}

// sort keys: Morton code of leaf low-corner cells, all ones for the rest
__global__ void k_oct_leafkeys(OctDev t, unsigned long long *__restrict__ key,
                               int *__restrict__ val, unsigned long long *__restrict__ nleaf) {
    const long long nc = (long long)t.nf * t.nf * t.nf;
    const long long c = blockIdx.x * (long long)OT + threadIdx.x;
    if (c >= nc) return;
    const int cx = (int)(c % t.nf), cy = (int)((c / t.nf) % t.nf), cz = (int)(c / ((long long)t.nf * t.nf));
    const int s = spc(t.Lmax, t.lev[c]);
    const bool low = (cx % s == 0) && (cy % s == 0) && (cz % s == 0);
    key[c] = low ? morton3(cx, cy, cz) : ~0ull;
    val[c] = (int)c;
    if (low) atomicAdd(nleaf, 1ull);
}

__global__ void k_oct_bricks(OctDev t, const int *__restrict__ cell_of_leaf, int4 *__restrict__ blow,
                             int *__restrict__ bmap) {
    const long long b = blockIdx.x * (long long)OT + threadIdx.x;
    if (b >= t.nb) return;
    const long long c = cell_of_leaf[b];
    const int cx = (int)(c % t.nf), cy = (int)((c / t.nf) % t.nf), cz = (int)(c / ((long long)t.nf * t.nf));
    const int l = t.lev[c];
    blow[b] = make_int4(cx * 8, cy * 8, cz * 8, l);
    const int f = spc(t.Lmax, l);
    for (int z = 0; z < f; ++z)
        for (int y = 0; y < f; ++y)
            for (int x = 0; x < f; ++x) bmap[cidx(t, cx + x, cy + y, cz + z)] = (int)b;
}

__global__ void k_oct_nbr(OctDev t, int *__restrict__ bnbr) {
    const long long b = blockIdx.x * (long long)OT + threadIdx.x;
    if (b >= t.nb) return;
    const int4 L = t.blow[b];
    const int S = spc(t.Lmax, L.w);  // finest-brick cells per side
    const int c0[3] = {L.x >> 3, L.y >> 3, L.z >> 3};
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1;
        int c[3] = {c0[0], c0[1], c0[2]};
        c[d] += (f & 1) ? S : -1;
        int r;
        if (c[d] < 0 || c[d] >= t.nf) {
            r = -2;
        } else {
            const int n = t.bmap[cidx(t, c[0], c[1], c[2])];
            r = t.blow[n].w == L.w ? n : -1;
        }
        bnbr[6 * b + f] = r;
    }
}

// pure row test (see the file header)
__device__ bool is_pure(const OctDev &t, const int P[3], int level) {
    const int s = spc(t.Lmax, level);
    for (int o = 0; o < 8; ++o) {
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = (P[d] - ((o >> d) & 1)) >> 3;
        if (t.lev[cidx(t, c[0], c[1], c[2])] != level) return false;
    }
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1;
        int Q[3] = {P[0], P[1], P[2]};
        Q[d] += (f & 1) ? s : -s;
        if (Q[d] == 0 || Q[d] == t.NL) continue;
        const int sq = touch_smax(t, Q[0], Q[1], Q[2]);
        if ((Q[0] % sq) || (Q[1] % sq) || (Q[2] % sq)) return false;
        const int b = t.bmap[cidx(t, Q[0] >> 3, Q[1] >> 3, Q[2] >> 3)];
        if (t.blow[b].w != level) return false;
    }
    return true;
}

// slot kinds and inside flags (from the finest-lattice classification)
__global__ void k_oct_slots(OctDev t, const uint8_t *__restrict__ vin, GridGeo vg,
                            uint8_t *__restrict__ inside, uint8_t *__restrict__ okind) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    int P[3], level;
    slot_pos(t, a, P, level);
    inside[a] = vin[((long long)P[2] * vg.ny + P[1]) * vg.nx + P[0]];
    int k = pos_kind(t, P[0], P[1], P[2]);
    uint8_t kind;
    if (k == 1) kind = 1;
    else if (k == 2) kind = 2;
    else kind = is_pure(t, P, level) ? 0 : 3;
    okind[a] = kind;
}

// listed edges of the finest lattice -> slot-based ids, and their +d end
__global__ void k_oct_cross_map(const long long *__restrict__ vid, long long nc, GridGeo vg,
                                OctDev t, unsigned long long *__restrict__ oid,
                                long long *__restrict__ slot_b, int *__restrict__ perm,
                                unsigned *__restrict__ err) {
    const long long s = blockIdx.x * (long long)OT + threadIdx.x;
    if (s >= nc) return;
    const long long id = vid[s];
    const int d = (int)(id / vg.N);
    const long long av = id - (long long)d * vg.N;
    int P[3] = {(int)(av % vg.nx), (int)((av / vg.nx) % vg.ny), (int)(av / ((long long)vg.nx * vg.ny))};
    const long long sa = owner_slot(t, P[0], P[1], P[2]);
    P[d] += 1;
    const long long sb = owner_slot(t, P[0], P[1], P[2]);
    bool ok = sa >= 0 && sb >= 0 && t.blow[sa >> 9].w == t.Lmax && t.blow[sb >> 9].w == t.Lmax;
    if (!ok) atomicOr(err, OERR_CROSS_OWNER);
    oid[s] = ok ? (unsigned long long)d * (unsigned long long)t.N + (unsigned long long)sa : ~0ull;
    slot_b[s] = sb;
    perm[s] = (int)s;
}

template <typename T>
__global__ void k_gather(const T *__restrict__ src, const int *__restrict__ perm, long long n,
                         int width, T *__restrict__ dst) {
    const long long q = blockIdx.x * (long long)OT + threadIdx.x;
    if (q >= n * width) return;
    const long long s = q / width;
    const int c = (int)(q - s * width);
    dst[q] = src[(long long)perm[s] * width + c];
}

__global__ void k_u64_to_i64(const unsigned long long *__restrict__ a, long long n,
                             long long *__restrict__ b) {
    const long long q = blockIdx.x * (long long)OT + threadIdx.x;
    if (q < n) b[q] = (long long)a[q];
}

__global__ void k_count_flags(const uint8_t *__restrict__ f, long long n, uint8_t val,
                              unsigned long long *__restrict__ out) {
    unsigned long long c = 0;
    for (long long q = blockIdx.x * (long long)OT + threadIdx.x; q < n; q += (long long)gridDim.x * OT)
        c += f[q] == val;
    using BR = cub::BlockReduce<unsigned long long, OT>;
    __shared__ typename BR::TempStorage tmp;
    c = BR(tmp).Sum(c);
    if (threadIdx.x == 0 && c) atomicAdd(out, c);
}

// ========================================================= coefficients ===
struct LevelConst {
    double h[8];     // cell size per level
    double kap[8];   // eps_out k_D^2 h^3 per level
    float w_in[8], w_out[8], kap32[8];
};

__global__ void k_oct_coef_pure(OctDev t, const uint8_t *__restrict__ inside, LevelConst lc,
                                double eps_in, double eps_out, double *__restrict__ W0,
                                double *__restrict__ W1, double *__restrict__ W2,
                                uint8_t *__restrict__ code) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    const int l = t.blow[a >> 9].w;
    const double w = (inside[a] ? eps_in : eps_out) * lc.h[l];
    W0[a] = w;
    W1[a] = w;
    W2[a] = w;
    code[a] = inside[a] ? 1 : 0;
}

// listed (finest) edges: Eq. WHA
__global__ void k_oct_coef_special(const long long *__restrict__ ids, const double *__restrict__ alpha,
                                   long long nc, long long N, double hf, double eps_in,
                                   double eps_out, double *__restrict__ W0, double *__restrict__ W1,
                                   double *__restrict__ W2, float *__restrict__ w0,
                                   float *__restrict__ w1, float *__restrict__ w2,
                                   uint8_t *__restrict__ code) {
    const long long s = blockIdx.x * (long long)OT + threadIdx.x;
    if (s >= nc) return;
    const int d = (int)(ids[s] / N);
    const long long a = ids[s] - (long long)d * N;
    const double al = alpha[s];
    const double w = 1.0 / (al / eps_in + (1.0 - al) / eps_out) * hf;
    double *W = d == 0 ? W0 : (d == 1 ? W1 : W2);
    float *w32 = d == 0 ? w0 : (d == 1 ? w1 : w2);
    W[a] = w;
    w32[a] = (float)w;
    // the three bits of one slot may be set by different threads
    unsigned *word = reinterpret_cast<unsigned *>(reinterpret_cast<uintptr_t>(code + a) & ~(uintptr_t)3);
    const int sh = 8 * (int)(reinterpret_cast<uintptr_t>(code + a) & 3);
    atomicOr(word, (2u << d) << sh);
}

// node kind into bits 4-5 of the code byte (read by the brick kernels)
__global__ void k_oct_code_kind(OctDev t, uint8_t *__restrict__ code) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a < t.N) code[a] = (uint8_t)((code[a] & 15) | (t.okind[a] << 4));
}

// neighbour slot of slot a (local loc) across direction f (-x,+x,-y,+y,-z,+z);
// -1 outside the domain or at a different level
__device__ __forceinline__ long long nbr_slot(const OctDev &t, long long a, int f) {
    const int loc = (int)(a & 511);
    const int i = loc & 7, j = (loc >> 3) & 7, k = loc >> 6;
    const long long b = a >> 9;
    switch (f) {
        case 0:
            if (i > 0) return a - 1;
            break;
        case 1:
            if (i < 7) return a + 1;
            break;
        case 2:
            if (j > 0) return a - 8;
            break;
        case 3:
            if (j < 7) return a + 8;
            break;
        case 4:
            if (k > 0) return a - 64;
            break;
        default:
            if (k < 7) return a + 64;
            break;
    }
    const int n = t.bnbr[6 * b + f];
    if (n < 0) return -1;
    const int wrap = (f == 0 ? 7 : f == 1 ? -7 : f == 2 ? 56 : f == 3 ? -56 : f == 4 ? 448 : -448);
    return ((long long)n << 9) + loc + wrap;
}

// FP64 diagonal of pure rows, in the order -x,+x,-y,+y,-z,+z then C
__global__ void k_oct_diag(OctDev t, const double *__restrict__ W0, const double *__restrict__ W1,
                           const double *__restrict__ W2, const uint8_t *__restrict__ inside,
                           LevelConst lc, double *__restrict__ diag) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    if (t.okind[a] != 0) {
        if (t.okind[a] != 3) diag[a] = 0.0;
        return;
    }
    const double *W[3] = {W0, W1, W2};
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        const long long m = nbr_slot(t, a, 2 * d);
        s = s + W[d][m];
        s = s + W[d][a];
    }
    const int l = t.blow[a >> 9].w;
    diag[a] = s + (inside[a] ? 0.0 : lc.kap[l]);
}

// ---------------------------------------------- level-transition rows ---
struct RowAcc {
    int col[MAXE];
    double val[MAXE];
    int n;
    double lift;
    unsigned err;
};

__device__ __forceinline__ void row_add(RowAcc &r, long long col, double v) {
    for (int q = 0; q < r.n; ++q)
        if (r.col[q] == (int)col) {
            r.val[q] += v;
            return;
        }
    if (r.n == MAXE) {
        r.err |= OERR_ROW_OVERFLOW;
        return;
    }
    r.col[r.n] = (int)col;
    r.val[r.n] = v;
    ++r.n;
}

// contribution v * x~(Q): a regular node is a column, a boundary node moves
// to the right-hand side, a hanging node spreads over its parents
__device__ void row_add_pos(const OctDev &t, const BcDesc &bd, RowAcc &r, const int Q[3], double v) {
    const int k = pos_kind(t, Q[0], Q[1], Q[2]);
    if (k == 0) {
        const long long c = owner_slot(t, Q[0], Q[1], Q[2]);
        row_add(r, c, v);
    } else if (k == 1) {
        r.lift -= v * bc_at(t, bd, Q);
    } else {
        int par[4][3];
        double w;
        const int np = hang_parents(t, Q, par, w);
        for (int q = 0; q < np; ++q) {
            const int pk = pos_kind(t, par[q][0], par[q][1], par[q][2]);
            if (pk == 0) {
                row_add(r, owner_slot(t, par[q][0], par[q][1], par[q][2]), v * w);
            } else if (pk == 1) {
                r.lift -= v * w * bc_at(t, bd, par[q]);
            } else {
                r.err |= OERR_HANGING_PARENT;
            }
        }
    }
}

__device__ bool pos_inside(const OctDev &t, const uint8_t *inside, const int P[3]) {
    const long long s = owner_slot(t, P[0], P[1], P[2]);
    return s >= 0 && inside[s];
}

// row of A = P^T K P for the regular node at P (a level-transition row);
// all nodes it touches are solvent
__device__ void transition_row(const OctDev &t, const BcDesc &bd, const uint8_t *inside,
                               const LevelConst &lc, double eps_out, const int P[3], RowAcc &r) {
    r.n = 0;
    r.lift = 0.0;
    r.err = 0;
    // rows of P^T that reach this node: itself and the hanging nodes it is a
    // parent of (at half the spacing of a touching leaf)
    int apos[MAXA][3];
    double aw[MAXA];
    int na = 0;
    apos[0][0] = P[0];
    apos[0][1] = P[1];
    apos[0][2] = P[2];
    aw[0] = 1.0;
    na = 1;
    int svals[2] = {0, 0}, ns = 0;
    for (int o = 0; o < 8; ++o) {
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = (P[d] - ((o >> d) & 1)) >> 3;
        const int s = spc(t.Lmax, t.lev[cidx(t, c[0], c[1], c[2])]);
        if (s < 2) continue;
        bool seen = false;
        for (int q = 0; q < ns; ++q) seen = seen || svals[q] == s;
        if (!seen && ns < 2) svals[ns++] = s;
    }
    for (int q = 0; q < ns; ++q) {
        const int half = svals[q] >> 1;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const int nz = (ox != 0) + (oy != 0) + (oz != 0);
                    if (nz == 0 || nz == 3) continue;
                    const int Q[3] = {P[0] + ox * half, P[1] + oy * half, P[2] + oz * half};
                    if (pos_kind(t, Q[0], Q[1], Q[2]) != 2) continue;
                    int smin;
                    const int sq = touch_spacings(t, Q[0], Q[1], Q[2], smin);
                    if (sq != svals[q]) continue;
                    // a node only if it lies on the lattice of a touching leaf
                    if ((Q[0] % smin) || (Q[1] % smin) || (Q[2] % smin)) continue;
                    const int off[3] = {ox, oy, oz};
                    bool match = true;
                    for (int d = 0; d < 3; ++d) match = match && ((Q[d] % sq != 0) == (off[d] != 0));
                    if (!match) continue;
                    if (na < MAXA) {
                        for (int d = 0; d < 3; ++d) apos[na][d] = Q[d];
                        aw[na] = 1.0 / (double)(1 << nz);
                        ++na;
                    } else {
                        r.err |= OERR_ROW_OVERFLOW;
                    }
                }
    }
    for (int qa = 0; qa < na; ++qa) {
        const int *A = apos[qa];
        const double wa = aw[qa];
        if (pos_inside(t, inside, A)) r.err |= OERR_SOLUTE_TRANSITION;
        double kaa = 0.0;
        for (int o = 0; o < 8; ++o) {
            int c[3], sg[3];
            for (int d = 0; d < 3; ++d) {
                sg[d] = ((o >> d) & 1) ? -1 : 1;
                c[d] = (A[d] - ((o >> d) & 1)) >> 3;
            }
            const int l = t.lev[cidx(t, c[0], c[1], c[2])];
            const int s = spc(t.Lmax, l);
            if ((A[0] % s) || (A[1] % s) || (A[2] % s)) continue;  // A is not a corner here
            const double we = (eps_out * lc.h[l]) * 0.25;
            for (int d = 0; d < 3; ++d) {
                int B[3] = {A[0], A[1], A[2]};
                B[d] += sg[d] * s;
                if (pos_inside(t, inside, B)) r.err |= OERR_SOLUTE_TRANSITION;
                kaa += we;
                row_add_pos(t, bd, r, B, -wa * we);
            }
            kaa += lc.kap[l] * 0.125;
        }
        row_add_pos(t, bd, r, A, wa * kaa);
    }
    // columns in increasing order
    for (int q = 1; q < r.n; ++q) {
        const int c = r.col[q];
        const double v = r.val[q];
        int p = q - 1;
        while (p >= 0 && r.col[p] > c) {
            r.col[p + 1] = r.col[p];
            r.val[p + 1] = r.val[p];
            --p;
        }
        r.col[p + 1] = c;
        r.val[p + 1] = v;
    }
}

__global__ void k_oct_tr_list(OctDev t, long long *__restrict__ counter, int *__restrict__ tr_slot) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    if (t.okind[a] == 3) {
        // compacted in any order here, sorted afterwards
        const long long q = atomicAdd((unsigned long long *)counter, 1ull);
        tr_slot[q] = (int)a;
    }
}

__global__ void k_oct_tr_rowmap(const int *__restrict__ tr_slot, long long ntr, int *__restrict__ tr_row) {
    const long long r = blockIdx.x * (long long)OT + threadIdx.x;
    if (r < ntr) tr_row[tr_slot[r]] = (int)r;
}

__global__ void __launch_bounds__(128)
k_oct_tr_count(OctDev t, BcDesc bd, const uint8_t *__restrict__ inside, LevelConst lc,
               double eps_out, const int *__restrict__ tr_slot, long long ntr,
               long long *__restrict__ nnz, unsigned *__restrict__ err) {
    const long long r = blockIdx.x * 128ll + threadIdx.x;
    if (r >= ntr) return;
    int P[3], level;
    slot_pos(t, tr_slot[r], P, level);
    RowAcc acc;
    BcDesc zero = bd;
    zero.kind = PB_BC_ZERO;  // counting needs no boundary values
    transition_row(t, zero, inside, lc, eps_out, P, acc);
    nnz[r] = acc.n;
    if (acc.err) atomicOr(err, acc.err);
}

__global__ void __launch_bounds__(128)
k_oct_tr_fill(OctDev t, BcDesc bd, const uint8_t *__restrict__ inside, LevelConst lc,
              double eps_out, const int *__restrict__ tr_slot, long long ntr,
              const long long *__restrict__ ptr, int *__restrict__ col, double *__restrict__ val,
              float *__restrict__ val32, double *__restrict__ tdiag, double *__restrict__ diag,
              double *__restrict__ lift) {
    const long long r = blockIdx.x * 128ll + threadIdx.x;
    if (r >= ntr) return;
    const long long a = tr_slot[r];
    int P[3], level;
    slot_pos(t, a, P, level);
    RowAcc acc;
    transition_row(t, bd, inside, lc, eps_out, P, acc);
    const long long p0 = ptr[r];
    double dg = 0.0;
    for (int q = 0; q < acc.n; ++q) {
        col[p0 + q] = acc.col[q];
        val[p0 + q] = acc.val[q];
        val32[p0 + q] = (float)acc.val[q];
        if (acc.col[q] == (int)a) dg = acc.val[q];
    }
    tdiag[r] = dg;
    diag[a] = dg;
    lift[r] = acc.lift;
}

// ================================================================ rhs ===
struct OTri {
    long long c[3];
    double w[3][2];
};

__device__ __forceinline__ OTri otri_cell(const GridGeo &g, double x, double y, double z) {
    OTri t;
    const double p[3] = {x, y, z};
    const long long nn[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) {
        const double u = (p[d] - g.o[d]) / g.h;
        long long c = (long long)floor(u);
        c = c < 0 ? 0 : (c > nn[d] - 2 ? nn[d] - 2 : c);
        const double tt = u - (double)c;
        t.c[d] = c;
        t.w[d][0] = 1.0 - tt;
        t.w[d][1] = tt;
    }
    return t;
}

// 4 pi l_B q trilinear deposit (Eq. RVop) on the finest cells: per (atom,
// corner), summed in increasing atom order by the smallest atom of a node
__global__ void k_oct_deposit(const double *__restrict__ atoms, long long na, GridGeo vg, OctDev t,
                              CellList cl, double coef0, double *__restrict__ f,
                              unsigned *__restrict__ err) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= 8 * na) return;
    const long long i = q >> 3;
    const int corner = (int)(q & 7);
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *Q = atoms + 4 * na;
    const OTri ti = otri_cell(vg, X[i], Y[i], Z[i]);
    const long long node[3] = {ti.c[0] + (corner & 1), ti.c[1] + ((corner >> 1) & 1),
                               ti.c[2] + ((corner >> 2) & 1)};
    double xa[3];
    int cc[3];
    for (int d = 0; d < 3; ++d) {
        xa[d] = vg.o[d] + (double)node[d] * vg.h;
        const double u = floor((xa[d] - cl.lo[d]) / cl.cs);
        cc[d] = (u < -4.0) ? -4 : ((u > (double)cl.dim[d] + 4.0) ? cl.dim[d] + 4 : (int)u);
    }
    constexpr int MAXC = 32;
    int ids[MAXC];
    int m = 0;
    for (int cz = cc[2] - 1; cz <= cc[2] + 1; ++cz) {
        if (cz < 0 || cz >= cl.dim[2]) continue;
        for (int cy = cc[1] - 1; cy <= cc[1] + 1; ++cy) {
            if (cy < 0 || cy >= cl.dim[1]) continue;
            for (int cx = cc[0] - 1; cx <= cc[0] + 1; ++cx) {
                if (cx < 0 || cx >= cl.dim[0]) continue;
                const int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
                for (int s = cl.start[cid]; s < cl.start[cid + 1]; ++s) {
                    const int j = cl.atom[s];
                    const OTri tj = (j == i) ? ti : otri_cell(vg, X[j], Y[j], Z[j]);
                    bool corner_of = true;
                    for (int d = 0; d < 3; ++d) {
                        const long long off = node[d] - tj.c[d];
                        if (off != 0 && off != 1) corner_of = false;
                    }
                    if (!corner_of) continue;
                    if (m < MAXC) {
                        int b = m - 1;
                        while (b >= 0 && ids[b] > j) {
                            ids[b + 1] = ids[b];
                            --b;
                        }
                        ids[b + 1] = j;
                        ++m;
                    }
                }
            }
        }
    }
    if (m == 0 || ids[0] != (int)i) return;
    double acc = 0.0;
    for (int qq = 0; qq < m; ++qq) {
        const int j = ids[qq];
        const OTri tj = (j == i) ? ti : otri_cell(vg, X[j], Y[j], Z[j]);
        const int dx = (int)(node[0] - tj.c[0]), dy = (int)(node[1] - tj.c[1]),
                  dz = (int)(node[2] - tj.c[2]);
        const double coef = coef0 * Q[j];
        acc = __dadd_rn(acc, __dmul_rn(coef, __dmul_rn(__dmul_rn(tj.w[0][dx], tj.w[1][dy]), tj.w[2][dz])));
    }
    const long long s = owner_slot(t, (int)node[0], (int)node[1], (int)node[2]);
    if (s < 0 || t.okind[s] != 0 || t.blow[s >> 9].w != t.Lmax) {
        atomicOr(err, OERR_DEPOSIT);
        return;
    }
    f[s] = acc;
}

// Dirichlet values at boundary slots; pure-row lift in the order -x,+x,-y,
// +y,-z,+z; transition rows add their own lift
__global__ void k_oct_bc(OctDev t, BcDesc bd, double *__restrict__ bc) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    if (t.okind[a] != 1) {
        bc[a] = 0.0;
        return;
    }
    int P[3], level;
    slot_pos(t, a, P, level);
    bc[a] = bc_at(t, bd, P);
}

__global__ void k_oct_lift(OctDev t, BcDesc bd, const double *__restrict__ W0,
                           const double *__restrict__ W1, const double *__restrict__ W2,
                           const double *__restrict__ bc, const int *__restrict__ tr_row,
                           const double *__restrict__ tlift, double *__restrict__ f) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    const uint8_t kd = t.okind[a];
    if (kd == 3) {
        f[a] += tlift[tr_row[a]];
        return;
    }
    if (kd != 0 || bd.kind == PB_BC_ZERO) return;
    int P[3], level;
    slot_pos(t, a, P, level);
    const int s = spc(t.Lmax, level);
    const double *W[3] = {W0, W1, W2};
    double v = f[a];
    for (int d = 0; d < 3; ++d) {
        if (P[d] - s == 0) v += W[d][nbr_slot(t, a, 2 * d)] * bc[nbr_slot(t, a, 2 * d)];
        if (P[d] + s == t.NL) {
            int Q[3] = {P[0], P[1], P[2]};
            Q[d] += s;
            v += W[d][a] * bc_at(t, bd, Q);
        }
    }
    f[a] = v;
}

// ======================================================== PCG kernels ===
// MODE_P: p = z + beta p_old, q = A p, sigma = p.q -> alpha
// MODE_U: q = A p, x += alpha p, z -= alpha q / D, rho = sum D z^2,
//         rr = sum (D z)^2 -> beta, stop test
// MODE_A: y = A x
enum { OM_P = 0, OM_U = 1, OM_A = 2 };

template <typename T>
struct OctArgs {
    OctDev t;
    const T *z, *pold;   // P
    T *p;                // P out, U in
    T *x, *zz;           // U in/out
    const T *xin;        // A in
    T *y;                // A out
    // compressed FP32 operator (pure rows)
    const uint8_t *code;
    const float *w32[3];
    // FP64 operator (pure rows)
    const double *W[3];
    const double *diag;
    LevelConst lc;
    // transition rows
    const int *tr_slot;
    const long long *tr_ptr;
    const int *tr_col;
    const T *tr_val;
    const double *tr_diag;
    long long ntr;
    CgState *st;
    double *partials;    // per-block slots of the dot products
};

template <int NT>
__device__ __forceinline__ double oblock_sum(double v, double *sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sred[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NT / 32; ++q) t += sred[q];
    return t;
}

// compensated FP32 sum (Neumaier): the value is s + c
__device__ __forceinline__ void onsum(float &s, float &c, float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
}
// the warp's compensated pairs combined in a fixed tree (lane 0 holds them)
__device__ __forceinline__ void owarp_nsum(float &s, float &c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        onsum(s, c, s2);
        c += c2;
    }
}

// FP32 form of olast_total below: each thread brings a compensated pair per
// value; warps, the block and then the last block over the per-block
// partials combine them compensated in FP32, in a fixed order (the last
// block runs alone at the end of the launch, and FP64 is a narrow pipe of
// GB300).  The totals (FP64) are valid in thread 0 of the last block.
template <int NT, int NV>
__device__ bool olast_total_f(unsigned *counter, float *partials, float (&s)[NV], float (&c)[NV],
                              double (&tot)[NV]) {
    __shared__ float sw[NT / 32][NV][2];
    __shared__ int s_last;
    const int nb = gridDim.x, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    auto block_pair = [&](int v, float &bs, float &bc) {
        bs = 0.f;
        bc = 0.f;
        for (int q = 0; q < NT / 32; ++q) {
            onsum(bs, bc, sw[q][v][0]);
            bc += sw[q][v][1];
        }
    };
#pragma unroll
    for (int v = 0; v < NV; ++v) owarp_nsum(s[v], c[v]);
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            sw[w][v][0] = s[v];
            sw[w][v][1] = c[v];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 0; v < NV; ++v) {
            float bs, bc;
            block_pair(v, bs, bc);
            partials[v * nb + blockIdx.x] = bs + bc;
        }
        __threadfence();
        s_last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int v = 0; v < NV; ++v) {
        float as = 0.f, ac = 0.f;
        for (int q = threadIdx.x; q < nb; q += NT) onsum(as, ac, __ldcg(partials + v * nb + q));
        owarp_nsum(as, ac);
        __syncthreads();
        if (l == 0) {
            sw[w][v][0] = as;
            sw[w][v][1] = ac;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float bs, bc;
            block_pair(v, bs, bc);
            tot[v] = (double)bs + (double)bc;
        }
    }
    return true;
}

// per-block partials then the last block's fixed-order total
template <int NT, int NV>
__device__ bool olast_total(unsigned *counter, double *partials, const double (&mine)[NV],
                            double (&tot)[NV]) {
    __shared__ double sred[NT / 32];
    __shared__ int s_last;
    const int nb = gridDim.x;
    double b[NV];
    for (int v = 0; v < NV; ++v) b[v] = oblock_sum<NT>(mine[v], sred);
    if (threadIdx.x == 0) {
        for (int v = 0; v < NV; ++v) partials[v * nb + blockIdx.x] = b[v];
        __threadfence();
        s_last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int v = 0; v < NV; ++v) {
        double a = 0.0;
        for (int q = threadIdx.x; q < nb; q += NT) a += __ldcg(partials + v * nb + q);
        tot[v] = oblock_sum<NT>(a, sred);
    }
    return true;
}

__device__ __forceinline__ void finalize_p(CgState *s, double t0) {
    s->sigma = t0;
    if (s->profile) {
        s->alpha = isfinite(t0) && t0 != 0.0 ? s->rho / t0 : 0.0;
    } else if (!(t0 > 0.0) || !isfinite(t0)) {
        s->done = 1;
        s->status = 1;
    } else {
        s->alpha = s->rho / t0;
    }
}

__device__ __forceinline__ void finalize_u(CgState *s, double t0, double t1) {
    s->beta = t0 / s->rho;
    s->rho = t0;
    s->rr = t1;
    s->iter += 1;
    if (s->profile) {
    } else if (!isfinite(t1)) {
        s->done = 1;
        s->status = 1;
    } else if (t1 <= s->rr_stop) {
        s->done = 1;
        s->status = 0;
    } else if (s->iter >= s->max_iter) {
        s->done = 1;
        s->status = 2;
    }
}

// Brick kernel of the pure rows.  A block works on four bricks at a time,
// 64 threads per brick, each thread owning the z-column (i, j) of its brick:
// the column's values stay in registers (its z neighbours), the brick's
// planes with their x/y face halos are staged in shared memory, and each
// brick's 64 threads synchronise on their own named barrier.  Only pure
// nodes are applied here; level-transition rows go to the CSR kernel.  Bits
// 4-5 of the code byte hold the node kind.  Dot products: FP32 within a
// brick, compensated FP32 across a thread's bricks and (in the FP32 solver)
// across threads and blocks, FP64 for the totals (GB300's FP64 rate is far
// below its FP32 rate).
constexpr int PX = 10;         // staged plane side (8 + 2 halo lines)
constexpr int PP = PX * PX;    // staged plane size

__device__ __forceinline__ void kahan(float &s, float &c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// 4-byte asynchronous copy global -> shared (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// named barrier of one 64-thread brick group (ids 1-4; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) {
    switch (g) {
        case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
        case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
        case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
        default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(OB, MODE == OM_U ? 3 : 4) k_oct_pure(OctArgs<T> A) {
    if (MODE != OM_A && *(volatile int *)&A.st->done) return;
    __shared__ T sv[4][8 * PP];
    __shared__ uint8_t sc[4][8 * PP];
    __shared__ int snb[4][6];
    // FP32 update kernel: the listed +x, +y, +z weights of each group's
    // brick (512 each), copied in asynchronously with the brick's values.
    // (The direction kernel keeps gathering them: the 15 KB more shared
    // memory per block, at its four blocks per SM, cost it more L1 than
    // the copies saved: 270 -> 290 us on the 20,000-atom octree, against
    // 331 -> 311 us for the update kernel.)
    constexpr bool F32 = sizeof(T) == 4;
    constexpr bool AW = F32 && MODE == OM_U;
    __shared__ float swt[AW ? 4 * 3 * 512 : 1];
    const OctDev &t = A.t;
    const int g = threadIdx.x >> 6, c = threadIdx.x & 63;
    const int i = c & 7, j = c >> 3;
    T beta = 0, alpha = 0;
    if (MODE == OM_P) beta = (T)A.st->beta;
    if (MODE == OM_U) alpha = (T)A.st->alpha;
    auto value = [&](int n, uint8_t cd) -> T {
        if (MODE == OM_P) return A.z[n] + beta * A.pold[n];
        if (MODE == OM_U) return A.p[n];
        return (cd >> 4) == 1 || (cd >> 4) == 2 ? (T)0 : A.xin[n];  // boundary entries read as zero
    };
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    double d0 = 0.0, d1 = 0.0;
    const int nb = (int)t.nb;
    T *V = sv[g];
    uint8_t *C = sc[g];
    const int q0 = (j + 1) * PX + (i + 1);  // this column's position in a staged plane
    // x/y face halos: 4 faces x 64 values, 4 per thread; f is this thread's face
    const int f = c >> 4;  // 0 -x, 1 +x, 2 -y, 3 +y
    // Neighbour ids are read one brick ahead, so that every global load of a
    // brick (own columns, face halos, z halos) issues before the first
    // shared-memory store and the brick waits on one memory latency, not two.
    const int bstride = gridDim.x * 4;
    int pf_f = -1, pf_zm = -1, pf_zp = -1, pf_s = -1;
    // (FP32) this column's code bytes are read one brick ahead too, so that
    // the brick's listed weights are copied in the same round trip as its
    // values instead of being gathered after the codes arrive
    unsigned long long pf_cd = 0ull;
    auto load_codes = [&](int bb) -> unsigned long long {
        unsigned long long w8 = 0ull;
        const int bs = (bb << 9) + c;
#pragma unroll
        for (int k = 0; k < 8; ++k) w8 |= (unsigned long long)A.code[bs + 64 * k] << (8 * k);
        return w8;
    };
    float *W1 = AW ? swt + g * 1536 : nullptr, *W3 = AW ? W1 + 512 : nullptr,
          *W5 = AW ? W1 + 1024 : nullptr;
    {
        const int b0 = blockIdx.x * 4 + g;
        if (b0 < nb) {
            pf_f = t.bnbr[6 * b0 + f];
            pf_zm = t.bnbr[6 * b0 + 4];
            pf_zp = t.bnbr[6 * b0 + 5];
            if (c < 6) pf_s = t.bnbr[6 * b0 + c];
            if constexpr (AW) pf_cd = load_codes(b0);
        }
    }
    for (int b = blockIdx.x * 4 + g; b < nb; b += bstride) {
        const int nbk = pf_f, nzm = pf_zm, nzp = pf_zp;
        group_sync(g);  // the group's previous brick is done with its buffers
        if (c < 6) snb[g][c] = pf_s;
        const unsigned long long cdw = pf_cd;
        if (b + bstride < nb) {
            const int bn = b + bstride;
            pf_f = t.bnbr[6 * bn + f];
            pf_zm = t.bnbr[6 * bn + 4];
            pf_zp = t.bnbr[6 * bn + 5];
            if (c < 6) pf_s = t.bnbr[6 * bn + c];
            if constexpr (AW) pf_cd = load_codes(bn);
        }
        const int level = t.blow[b].w;
        T wi = 0, wo = 0, kp = 0;
        if constexpr (sizeof(T) == 4) {
            wi = A.lc.w_in[level];
            wo = A.lc.w_out[level];
            kp = A.lc.kap32[level];
        }
        const int base = (b << 9) + c;
        T v[8], xr[MODE == OM_U ? 8 : 1], zr[MODE == OM_U ? 8 : 1];
        uint8_t cd[8];
        if constexpr (AW) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                cd[k] = (uint8_t)(cdw >> (8 * k));
                const int a = base + 64 * k;
                if (cd[k] & 2) cp_async4(W1 + 64 * k + c, A.w32[0] + a);
                if (cd[k] & 4) cp_async4(W3 + 64 * k + c, A.w32[1] + a);
                if (cd[k] & 8) cp_async4(W5 + 64 * k + c, A.w32[2] + a);
            }
            cp_async_commit();
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (!AW) cd[k] = A.code[base + 64 * k];
            v[k] = value(base + 64 * k, cd[k]);
            if constexpr (MODE == OM_U) {
                xr[k] = A.x[base + 64 * k];
                zr[k] = A.zz[base + 64 * k];
            }
        }
        T hv[4];
        uint8_t hc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = (c & 15) + 16 * r;
            const int u = m & 7, k = m >> 3;
            int n = f < 2 ? (k * 8 + u) * 8 + (f == 0 ? 7 : 0) : (k * 8 + (f == 2 ? 7 : 0)) * 8 + u;
            hv[r] = 0;
            hc[r] = 0;
            if (nbk >= 0) {
                n += nbk << 9;
                hc[r] = A.code[n];
                hv[r] = value(n, hc[r]);
            }
        }
        // z halos of this column and the -z neighbour's code
        T zm = 0, zp = 0;
        uint8_t czm = 0;
        if (nzm >= 0) {
            const int n = (nzm << 9) + 448 + c;
            czm = A.code[n];
            zm = value(n, czm);
        }
        if (nzp >= 0) zp = value((nzp << 9) + c, A.code[(nzp << 9) + c]);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            V[k * PP + q0] = v[k];
            C[k * PP + q0] = cd[k];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = (c & 15) + 16 * r;
            const int u = m & 7, k = m >> 3;
            const int sq = f < 2 ? k * PP + (u + 1) * PX + (f == 0 ? 0 : 9)
                                 : k * PP + (f == 2 ? 0 : 9) * PX + (u + 1);
            V[sq] = hv[r];
            C[sq] = hc[r];
        }
        if constexpr (AW) cp_async_wait_all();
        group_sync(g);  // staged planes, weights and snb visible
        float bs0 = 0.f, bs1 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = base + 64 * k;
            const uint8_t cc = cd[k];
            const int kind = cc >> 4;
            if (kind != 0) {
                if (MODE == OM_A && kind != 3) A.y[a] = (T)0;
                continue;
            }
            const int q = k * PP + q0;
            const T xm = V[q - 1], xp = V[q + 1], ym = V[q - PX], yp = V[q + PX];
            const T zmv = k > 0 ? v[k - 1] : zm, zpv = k < 7 ? v[k + 1] : zp;
            T w[6];  // -x, +x, -y, +y, -z, +z
            if constexpr (sizeof(T) == 4) {
                const uint8_t cxm = C[q - 1], cym = C[q - PX];
                const uint8_t czmk = k > 0 ? cd[k - 1] : czm;
                const T wself = (cc & 1) ? wi : wo;
                if constexpr (AW) {
                    // listed weights of the brick's own edges from shared
                    // memory, of edges into a neighbouring brick gathered
                    w[1] = (cc & 2) ? W1[64 * k + c] : wself;
                    w[3] = (cc & 4) ? W3[64 * k + c] : wself;
                    w[5] = (cc & 8) ? W5[64 * k + c] : wself;
                    if (cxm & 2)
                        w[0] = i > 0 ? W1[64 * k + c - 1]
                                     : A.w32[0][(snb[g][0] << 9) + (a & 511) + 7];
                    else
                        w[0] = (cxm & 1) ? wi : wo;
                    if (cym & 4)
                        w[2] = j > 0 ? W3[64 * k + c - 8]
                                     : A.w32[1][(snb[g][2] << 9) + (a & 511) + 56];
                    else
                        w[2] = (cym & 1) ? wi : wo;
                    if (czmk & 8)
                        w[4] = k > 0 ? W5[64 * (k - 1) + c]
                                     : A.w32[2][(nzm << 9) + (a & 511) + 448];
                    else
                        w[4] = (czmk & 1) ? wi : wo;
                } else {
                    w[1] = (cc & 2) ? A.w32[0][a] : wself;
                    w[3] = (cc & 4) ? A.w32[1][a] : wself;
                    w[5] = (cc & 8) ? A.w32[2][a] : wself;
                    if (cxm & 2) w[0] = A.w32[0][i > 0 ? a - 1 : (snb[g][0] << 9) + (a & 511) + 7];
                    else w[0] = (cxm & 1) ? wi : wo;
                    if (cym & 4) w[2] = A.w32[1][j > 0 ? a - 8 : (snb[g][2] << 9) + (a & 511) + 56];
                    else w[2] = (cym & 1) ? wi : wo;
                    if (czmk & 8) w[4] = A.w32[2][k > 0 ? a - 64 : (nzm << 9) + (a & 511) + 448];
                    else w[4] = (czmk & 1) ? wi : wo;
                }
            } else {
                w[0] = A.W[0][i > 0 ? a - 1 : (snb[g][0] << 9) + (a & 511) + 7];
                w[1] = A.W[0][a];
                w[2] = A.W[1][j > 0 ? a - 8 : (snb[g][2] << 9) + (a & 511) + 56];
                w[3] = A.W[1][a];
                w[4] = A.W[2][k > 0 ? a - 64 : (nzm << 9) + (a & 511) + 448];
                w[5] = A.W[2][a];
            }
            const T sum = w[0] * xm + w[1] * xp + w[2] * ym + w[3] * yp + w[4] * zmv + w[5] * zpv;
            T D;
            if constexpr (sizeof(T) == 4) {
                D = (((((w[0] + w[1]) + w[2]) + w[3]) + w[4]) + w[5]) + ((cc & 1) ? (T)0 : kp);
            } else {
                D = A.diag[a];
            }
            const T pa = v[k];
            const T qv = D * pa - sum;
            if (MODE == OM_P) {
                A.p[a] = pa;
                if constexpr (sizeof(T) == 4) bs0 += pa * qv;
                else d0 += pa * qv;
            } else if (MODE == OM_U) {
                A.x[a] = xr[k] + alpha * pa;
                T zn;
                if constexpr (sizeof(T) == 4) zn = zr[k] - __fdividef(alpha * qv, D);
                else zn = zr[k] - alpha * qv / D;
                A.zz[a] = zn;
                const T dz = D * zn;
                if constexpr (sizeof(T) == 4) {
                    bs0 += dz * zn;
                    bs1 += dz * dz;
                } else {
                    d0 += dz * zn;
                    d1 += dz * dz;
                }
            } else {
                A.y[a] = qv;
            }
        }
        if constexpr (sizeof(T) == 4) {
            kahan(s0, c0, bs0);
            kahan(s1, c1, bs1);
        }
    }
    // level-transition rows (explicit CSR): each block takes a fixed
    // contiguous range of rows, one row per thread at a time (rows r0 + tid,
    // + OB, + 2 OB, ...).  The bounds of the row after next are read, and
    // the next row's entries brought into L1, while a row is summed, so a
    // row waits on its value gathers only.
    if (A.ntr > 0) {
        const long long per = (A.ntr + gridDim.x - 1) / gridDim.x;
        const long long r0 = (long long)blockIdx.x * per;
        const long long r1 = min(A.ntr, r0 + per);
        long long na0 = 0, na1 = 0, nb0 = 0, nb1 = 0;  // bounds of rows r + OB, r + 2 OB
        {
            const long long r = r0 + threadIdx.x;
            if (r < r1) {
                na0 = A.tr_ptr[r];
                na1 = A.tr_ptr[r + 1];
            }
            if (r + OB < r1) {
                nb0 = A.tr_ptr[r + OB];
                nb1 = A.tr_ptr[r + OB + 1];
            }
        }
        for (long long r = r0 + threadIdx.x; r < r1; r += OB) {
            const long long e0 = na0, e1 = na1;
            na0 = nb0;
            na1 = nb1;
            if (r + 2 * OB < r1) {
                nb0 = A.tr_ptr[r + 2 * OB];
                nb1 = A.tr_ptr[r + 2 * OB + 1];
            }
            if (r + OB < r1 && na1 > na0) {
                asm volatile("prefetch.global.L1 [%0];" ::"l"(A.tr_col + na0));
                asm volatile("prefetch.global.L1 [%0];" ::"l"(A.tr_val + na0));
            }
            const int a = A.tr_slot[r];
            T q = 0;
            for (long long e = e0; e < e1; ++e) {
                const int c = A.tr_col[e];
                T v;
                if (MODE == OM_P) v = A.z[c] + beta * A.pold[c];
                else if (MODE == OM_U) v = A.p[c];
                else v = A.xin[c];
                q += A.tr_val[e] * v;
            }
            if (MODE == OM_P) {
                const T pa = A.z[a] + beta * A.pold[a];
                A.p[a] = pa;
                if constexpr (sizeof(T) == 4) kahan(s0, c0, pa * q);
                else d0 += pa * q;
            } else if (MODE == OM_U) {
                const T D = (T)A.tr_diag[r];
                const T pa = A.p[a];
                A.x[a] += alpha * pa;
                const T zn = A.zz[a] - alpha * q / D;
                A.zz[a] = zn;
                const T dz = D * zn;
                if constexpr (sizeof(T) == 4) {
                    kahan(s0, c0, dz * zn);
                    kahan(s1, c1, dz * dz);
                } else {
                    d0 += dz * zn;
                    d1 += dz * dz;
                }
            } else {
                A.y[a] = q;
            }
        }
    }
    if (MODE == OM_A) return;
    auto finish = [&](const double (&tot)[2]) {
        CgState *s = A.st;
        if (MODE == OM_P) {
            finalize_p(s, tot[0]);
        } else {
            finalize_u(s, tot[0], tot[1]);
        }
        s->counter = 0;
    };
    double tot[2];
    if constexpr (sizeof(T) == 4) {
        // Kahan pairs (value s - c) as compensated pairs (value s + c')
        float ps[2] = {s0, s1}, pc[2] = {-c0, -c1};
        if (olast_total_f<OB, 2>(&A.st->counter, reinterpret_cast<float *>(A.partials), ps, pc,
                                 tot) &&
            threadIdx.x == 0)
            finish(tot);
    } else {
        double mine[2] = {d0, d1};
        if (olast_total<OB, 2>(&A.st->counter, A.partials, mine, tot) && threadIdx.x == 0)
            finish(tot);
    }
}

// FP64 true residual r = f - A x (x = phi on the unknowns), z = r / D in
// the inner solver's precision; |r|^2 and r.z to the CG state
template <typename TZ>
__global__ void __launch_bounds__(OT)
k_oct_residual(OctDev t, const double *__restrict__ phi, const double *__restrict__ f,
               const double *__restrict__ W0, const double *__restrict__ W1,
               const double *__restrict__ W2, const double *__restrict__ diag,
               const int *__restrict__ tr_row, const long long *__restrict__ tr_ptr,
               const int *__restrict__ tr_col, const double *__restrict__ tr_val,
               TZ *__restrict__ zout, CgState *st, double *partials) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    double rr = 0.0, rz = 0.0;
    if (a < t.N) {
        const uint8_t kd = t.okind[a];
        if (kd == 0 || kd == 3) {
            double s;
            if (kd == 0) {
                const double *W[3] = {W0, W1, W2};
                s = diag[a] * phi[a];
                for (int d = 0; d < 3; ++d) {
                    const long long m = nbr_slot(t, a, 2 * d), pn = nbr_slot(t, a, 2 * d + 1);
                    if (m >= 0 && t.okind[m] != 1) s -= W[d][m] * phi[m];
                    if (pn >= 0 && t.okind[pn] != 1) s -= W[d][a] * phi[pn];
                }
            } else {
                const int r = tr_row[a];
                s = 0.0;
                for (long long e = tr_ptr[r]; e < tr_ptr[r + 1]; ++e) s += tr_val[e] * phi[tr_col[e]];
            }
            const double r = f[a] - s;
            TZ z;
            if (sizeof(TZ) == 4) z = (TZ)((float)r / (float)diag[a]);
            else z = (TZ)(r / diag[a]);
            zout[a] = z;
            rr = r * r;
            rz = r * (double)z;
        }
    }
    double mine[2] = {rr, rz}, tot[2];
    if (olast_total<OT, 2>(&st->counter, partials, mine, tot)) {
        if (threadIdx.x == 0) {
            st->res64 = tot[0];
            st->rz64 = tot[1];
            st->counter = 0;
        }
    }
}

template <typename TX>
__global__ void k_oct_promote(OctDev t, double *__restrict__ phi, const TX *__restrict__ x) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    const uint8_t kd = t.okind[a];
    if (kd == 0 || kd == 3) phi[a] += (double)x[a];
}

// phi at hanging slots from their parents (output only)
__global__ void k_oct_hang(OctDev t, BcDesc bd, double *__restrict__ phi) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N || t.okind[a] != 2) return;
    int P[3], level;
    slot_pos(t, a, P, level);
    int par[4][3];
    double w;
    const int np = hang_parents(t, P, par, w);
    double v = 0.0;
    for (int q = 0; q < np; ++q) {
        const long long s = owner_slot(t, par[q][0], par[q][1], par[q][2]);
        v += w * (s >= 0 ? phi[s] : bc_at(t, bd, par[q]));
    }
    phi[a] = v;
}

__global__ void k_oct_kappa(OctDev t, const uint8_t *__restrict__ inside, LevelConst lc,
                            double *__restrict__ out) {
    const long long a = blockIdx.x * (long long)OT + threadIdx.x;
    if (a >= t.N) return;
    out[a] = inside[a] ? 0.0 : lc.kap[t.blow[a >> 9].w];
}

// ============================================================= energy ===
constexpr int EN_T = 256;

__global__ void __launch_bounds__(EN_T)
k_oct_energy(const long long *__restrict__ ids, const long long *__restrict__ slot_b,
             const double *__restrict__ alpha, const int8_t *__restrict__ sign, long long ncross,
             long long N, const double *__restrict__ W0, const double *__restrict__ W1,
             const double *__restrict__ W2, const double *__restrict__ phi,
             const double *__restrict__ Phi, const double *__restrict__ Psi,
             const double *__restrict__ Tw, const double *__restrict__ PsiN, double h,
             double eps_in, double eps_out, double lB, double *partials, EnergyAcc *acc) {
    double S = 0.0, I = 0.0, F = 0.0, Im = 0.0;
    for (long long s = blockIdx.x * (long long)EN_T + threadIdx.x; s < ncross;
         s += (long long)gridDim.x * EN_T) {
        const int sg = sign[s];
        if (sg == 0) continue;
        const int d = (int)(ids[s] / N);
        const long long a = ids[s] - (long long)d * N, b = slot_b[s];
        const double *W = d == 0 ? W0 : (d == 1 ? W1 : W2);
        const long long in = sg > 0 ? a : b, out = sg > 0 ? b : a;
        const double pin = phi[in], pout = phi[out];
        const double Fe = W[a] * (pin - pout);
        const double al = alpha[s];
        const double phip = pin + (al / eps_in) * (pout - pin) / (al / eps_in + (1.0 - al) / eps_out);
        S += Fe * Phi[s];
        I += phip * (h * h) * Psi[s];
        F += Fe;
        Im += Tw[s] * phip * PsiN[s];
    }
    double mine[4] = {S, I, F, Im}, tot[4];
    if (olast_total<EN_T, 4>(&acc->counter, partials, mine, tot)) {
        if (threadIdx.x == 0) {
            const double fourpi = 4.0 * M_PI;
            acc->S = tot[0];
            acc->I = tot[1];
            acc->F = tot[2];
            acc->Imc = tot[3];
            pb_energy_terms o{};
            o.e_coul = (lB / eps_in) * 0.5 * acc->ecoul_sum;
            o.e_pol = 0.5 * (1.0 / eps_out - 1.0 / eps_in) * tot[0] / fourpi;
            o.e_ion_flux = -0.5 * (1.0 / eps_out) * tot[0] / fourpi;
            o.e_ion_surf = 0.5 * tot[1] / fourpi;
            o.e_total = o.e_coul + o.e_pol + o.e_ion_surf + o.e_ion_flux;
            o.flux_charge = tot[2] / (fourpi * lB);
            o.e_ion_mc = 0.5 * tot[3] / fourpi;
            acc->out = o;
            acc->counter = 0;
        }
    }
}

// ============================================================== host ===
double wall_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

LevelConst level_const(const pb_system *sys) {
    const OctDev &t = sys->g->ot;
    LevelConst lc{};
    for (int l = 0; l <= t.Lmax && l < 8; ++l) {
        const double h = t.hf * (double)spc(t.Lmax, l);
        lc.h[l] = h;
        lc.kap[l] = sys->p.eps_out * sys->kD * sys->kD * h * h * h;
        lc.w_in[l] = (float)(sys->p.eps_in * h);
        lc.w_out[l] = (float)(sys->p.eps_out * h);
        lc.kap32[l] = (float)lc.kap[l];
    }
    return lc;
}

BcDesc bc_desc(const pb_system *sys) {
    BcDesc bd;
    bd.atoms = sys->g->atoms;
    bd.na = sys->g->na;
    bd.scale = sys->lB / sys->p.eps_out;
    bd.k = sys->p.bc == PB_BC_DH ? sys->kD : 0.0;
    bd.kind = sys->p.bc;
    return bd;
}

// persistent grid of a brick kernel: its resident blocks per SM x SMs
template <typename T, int MODE>
int pure_grid() {
    static int g = 0;
    if (!g) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_oct_pure<T, MODE>, OB, 0) !=
                cudaSuccess ||
            per <= 0) {
            cudaGetLastError();
            per = 3;
        }
        g = per * num_sms();
    }
    return g;
}

}  // namespace

// ------------------------------------------------------------- build ---
pb_status oct_build(pb_grid *g, const pb_grid_spec *spec, cudaStream_t s) {
    const long long na = g->na;
    const double hf = spec->h_fine, hb = spec->h_bulk, dist = spec->refine_dist;
    int Lmax = 0;
    while (Lmax < 7 && hf * (double)(1 << Lmax) < hb) ++Lmax;
    if (!(hf > 0.0) || hf * (double)(1 << Lmax) != hb) {
        set_error("octree: h_bulk must be h_fine times a power of two (at most 2^7)");
        return PB_ERR_ARG;
    }
    // bounding box, radii
    PB_CUDA_TRY(cudaMemsetAsync(g->d_info, 0, sizeof(BuildInfo), s));
    k_oct_bbox<<<1, OT, 0, s>>>(g->atoms, na, g->d_info);
    PB_LAUNCH_CHECK();
    BuildInfo hinfo;
    PB_CUDA_TRY(cudaMemcpyAsync(&hinfo, g->d_info, sizeof(BuildInfo), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo.err & ERRF_ATOM_VALUE) {
        set_error("atoms: non-finite value or non-positive radius");
        return PB_ERR_ARG;
    }
    // de-refined domain: levels coarser than h_tight are split inside the tight box
    int Lt = 0;
    double h_near = hb;
    if (spec->h_tight > 0.0) {
        while (Lt < Lmax && spec->h_tight * (double)(1 << Lt) < hb) ++Lt;
        if (spec->h_tight * (double)(1 << Lt) != hb || !(spec->tight_fill >= 1.0)) {
            set_error("octree: h_bulk must be h_tight times a power of two, h_tight at least "
                      "h_fine, and tight_fill at least 1");
            return PB_ERR_ARG;
        }
        h_near = spec->h_tight;
    }
    if (!(dist >= hinfo.rmax) || !(dist >= hf) || !(dist >= 1.5 * h_near)) {
        set_error("octree: refine_dist must be at least the largest radius, h_fine and 1.5 h_bulk "
                  "(1.5 h_tight on a de-refined domain)");
        return PB_ERR_ARG;
    }
    double3 tlo = make_double3(0.0, 0.0, 0.0), thi = tlo;
    if (Lt > 0) {
        double ext = 0.0;
        for (int d = 0; d < 3; ++d) ext = std::max(ext, hinfo.hi[d] - hinfo.lo[d]);
        const double half = 0.5 * spec->tight_fill * ext;
        tlo = make_double3(0.5 * (hinfo.lo[0] + hinfo.hi[0]) - half,
                           0.5 * (hinfo.lo[1] + hinfo.hi[1]) - half,
                           0.5 * (hinfo.lo[2] + hinfo.hi[2]) - half);
        thi = make_double3(0.5 * (hinfo.lo[0] + hinfo.hi[0]) + half,
                           0.5 * (hinfo.lo[1] + hinfo.hi[1]) + half,
                           0.5 * (hinfo.lo[2] + hinfo.hi[2]) + half);
    }
    OctDev &t = g->ot;
    t.hf = hf;
    t.Lmax = Lmax;
    if (spec->n[0] > 0) {
        t.n0 = spec->n[0];
        for (int d = 0; d < 3; ++d) t.o[d] = spec->origin[d];
    } else {
        double ext = 0.0;
        for (int d = 0; d < 3; ++d) ext = std::max(ext, hinfo.hi[d] - hinfo.lo[d]);
        t.n0 = std::max(1, (int)ceil(spec->fill * ext / (8.0 * hb)));
        const double side = (double)t.n0 * 8.0 * hb;
        for (int d = 0; d < 3; ++d) t.o[d] = 0.5 * (hinfo.lo[d] + hinfo.hi[d]) - 0.5 * side;
    }
    t.nf = t.n0 << Lmax;
    t.NL = 8 * t.nf;
    if (t.NL + 1 > 1290) {
        set_error("octree: the finest lattice has more than 1290 nodes per axis");
        return PB_ERR_ARG;
    }
    // uniform pass on the finest lattice: classification, cell list, listed edges
    pb_grid_spec vs{};
    vs.kind = PB_GRID_UNIFORM;
    for (int d = 0; d < 3; ++d) {
        vs.n[d] = t.NL + 1;
        vs.origin[d] = t.o[d];
    }
    vs.h = hf;
    pb_status rc = grid_build(g, &vs, s);
    if (rc != PB_OK) return rc;
    g->vgeo = g->geo;
    const GridGeo vg = g->vgeo;

    // refinement levels
    const long long nc = (long long)t.nf * t.nf * t.nf;
    std::vector<uint8_t *> near(Lmax, nullptr), split(Lmax, nullptr);
    t.lev = (uint8_t *)dalloc(nc, s);
    t.bmap = (int *)dalloc(sizeof(int) * nc, s);
    uint8_t *req = (uint8_t *)dalloc(nc, s);
    int *changed = (int *)dalloc(sizeof(int) * 2, s);
    if (!t.lev || !t.bmap || !req || !changed) return PB_ERR_OOM;
    LevelPtrs np{}, sp{};
    for (int l = 0; l < Lmax; ++l) {
        const long long nl = (long long)t.n0 << l;
        near[l] = (uint8_t *)dalloc(nl * nl * nl, s);
        split[l] = (uint8_t *)dalloc(nl * nl * nl, s);
        if (!near[l] || !split[l]) return PB_ERR_OOM;
        k_oct_near<<<cdiv(nl * nl * nl, OT), OT, 0, s>>>(g->atoms, na, t, l, dist,
                                                          hinfo.rmax + dist, g->cells,
                                                          l > 0 ? near[l - 1] : nullptr, near[l],
                                                          l < Lt, tlo, thi);
        PB_LAUNCH_CHECK();
        np.p[l] = near[l];
        sp.p[l] = split[l];
    }
    k_oct_levels<<<cdiv(nc, OT), OT, 0, s>>>(t, np, t.lev);
    PB_LAUNCH_CHECK();
    for (int it = 0; it < 64; ++it) {
        PB_CUDA_TRY(cudaMemsetAsync(changed, 0, sizeof(int), s));
        k_oct_req<<<cdiv(nc, OT), OT, 0, s>>>(t, t.lev, req);
        PB_LAUNCH_CHECK();
        for (int l = 0; l < Lmax; ++l) {
            const long long nl = (long long)t.n0 << l;
            k_oct_split<<<cdiv(nl * nl * nl, OT), OT, 0, s>>>(t, l, req, split[l]);
            PB_LAUNCH_CHECK();
        }
        k_oct_relevel<<<cdiv(nc, OT), OT, 0, s>>>(t, sp, t.lev, changed);
        PB_LAUNCH_CHECK();
        int hc = 0;
        PB_CUDA_TRY(cudaMemcpyAsync(&hc, changed, sizeof(int), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        if (!hc) break;
        if (it == 63) {
            set_error("octree: 2:1 balance did not settle");
            return PB_ERR_CUDA;
        }
    }
    for (int l = 0; l < Lmax; ++l) {
        dfree(near[l], s);
        dfree(split[l], s);
    }
    dfree(req, s);

    // leaves in Morton order
    unsigned long long *keys = (unsigned long long *)dalloc(sizeof(unsigned long long) * nc, s);
    unsigned long long *keys2 = (unsigned long long *)dalloc(sizeof(unsigned long long) * nc, s);
    int *vals = (int *)dalloc(sizeof(int) * nc, s);
    int *vals2 = (int *)dalloc(sizeof(int) * nc, s);
    unsigned long long *cnt = (unsigned long long *)dalloc(sizeof(unsigned long long) * 2, s);
    if (!keys || !keys2 || !vals || !vals2 || !cnt) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2, s));
    k_oct_leafkeys<<<cdiv(nc, OT), OT, 0, s>>>(t, keys, vals, cnt);
    PB_LAUNCH_CHECK();
    size_t tb = 0;
    PB_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, keys, keys2, vals, vals2, (int)nc, 0, 64, s));
    void *tmp = dalloc(tb, s);
    if (!tmp) return PB_ERR_OOM;
    PB_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, keys, keys2, vals, vals2, (int)nc, 0, 64, s));
    note_launch(4);
    unsigned long long hnb = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&hnb, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(tmp, s);
    t.nb = (long long)hnb;
    t.N = t.nb * 512;
    if (t.N > (1ll << 31) - 1) {
        set_error("octree: more than 2^31 node slots");
        return PB_ERR_ARG;
    }
    t.blow = (int4 *)dalloc(sizeof(int4) * t.nb, s);
    t.bnbr = (int *)dalloc(sizeof(int) * 6 * t.nb, s);
    t.okind = (uint8_t *)dalloc(t.N, s);
    uint8_t *sin = (uint8_t *)dalloc(t.N, s);
    if (!t.blow || !t.bnbr || !t.okind || !sin) return PB_ERR_OOM;
    k_oct_bricks<<<cdiv(t.nb, OT), OT, 0, s>>>(t, vals2, t.blow, t.bmap);
    PB_LAUNCH_CHECK();
    dfree(keys, s);
    dfree(keys2, s);
    dfree(vals, s);
    dfree(vals2, s);
    k_oct_nbr<<<cdiv(t.nb, OT), OT, 0, s>>>(t, t.bnbr);
    PB_LAUNCH_CHECK();
    k_oct_slots<<<cdiv(t.N, OT), OT, 0, s>>>(t, g->inside, vg, sin, t.okind);
    PB_LAUNCH_CHECK();

    // listed edges renumbered by slot, in increasing order
    unsigned *err = (unsigned *)dalloc(sizeof(unsigned), s);
    if (!err) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    const long long ncr = g->ncross;
    long long ncr1 = ncr > 0 ? ncr : 1;
    g->cslot_b = (long long *)dalloc(sizeof(long long) * ncr1, s);
    if (!g->cslot_b) return PB_ERR_OOM;
    if (ncr > 0) {
        unsigned long long *oid = (unsigned long long *)dalloc(sizeof(unsigned long long) * ncr, s);
        unsigned long long *oid2 = (unsigned long long *)dalloc(sizeof(unsigned long long) * ncr, s);
        int *perm = (int *)dalloc(sizeof(int) * ncr, s);
        int *perm2 = (int *)dalloc(sizeof(int) * ncr, s);
        long long *sb = (long long *)dalloc(sizeof(long long) * ncr, s);
        double *al2 = (double *)dalloc(sizeof(double) * ncr, s);
        double *rp2 = (double *)dalloc(sizeof(double) * 3 * ncr, s);
        int8_t *sg2 = (int8_t *)dalloc(ncr, s);
        if (!oid || !oid2 || !perm || !perm2 || !sb || !al2 || !rp2 || !sg2) return PB_ERR_OOM;
        k_oct_cross_map<<<cdiv(ncr, OT), OT, 0, s>>>(g->cid, ncr, vg, t, oid, sb, perm, err);
        PB_LAUNCH_CHECK();
        tb = 0;
        PB_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, oid, oid2, perm, perm2, (int)ncr, 0, 64, s));
        tmp = dalloc(tb, s);
        if (!tmp) return PB_ERR_OOM;
        PB_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tb, oid, oid2, perm, perm2, (int)ncr, 0, 64, s));
        note_launch(4);
        k_u64_to_i64<<<cdiv(ncr, OT), OT, 0, s>>>(oid2, ncr, g->cid);
        k_gather<double><<<cdiv(ncr, OT), OT, 0, s>>>(g->calpha, perm2, ncr, 1, al2);
        k_gather<double><<<cdiv(3 * ncr, OT), OT, 0, s>>>(g->crp, perm2, ncr, 3, rp2);
        k_gather<int8_t><<<cdiv(ncr, OT), OT, 0, s>>>(g->csign, perm2, ncr, 1, sg2);
        k_gather<long long><<<cdiv(ncr, OT), OT, 0, s>>>(sb, perm2, ncr, 1, g->cslot_b);
        PB_LAUNCH_CHECK();
        note_launch(4);
        // the re-triangulated surface of the finest lattice, in the new order
        double *mw2 = (double *)dalloc(sizeof(double) * ncr, s);
        double *mn2 = (double *)dalloc(sizeof(double) * 3 * ncr, s);
        if (!mw2 || !mn2) return PB_ERR_OOM;
        k_gather<double><<<cdiv(ncr, OT), OT, 0, s>>>(g->mc_w, perm2, ncr, 1, mw2);
        k_gather<double><<<cdiv(3 * ncr, OT), OT, 0, s>>>(g->mc_n, perm2, ncr, 3, mn2);
        PB_LAUNCH_CHECK();
        note_launch(1);
        dfree(g->mc_w, s);
        dfree(g->mc_n, s);
        g->mc_w = mw2;
        g->mc_n = mn2;
        dfree(tmp, s);
        dfree(oid, s);
        dfree(oid2, s);
        dfree(perm, s);
        dfree(perm2, s);
        dfree(sb, s);
        dfree(g->calpha, s);
        dfree(g->crp, s);
        dfree(g->csign, s);
        g->calpha = al2;
        g->crp = rp2;
        g->csign = sg2;
    }
    // inside count of the slots
    PB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2, s));
    k_count_flags<<<num_sms() * 4, OT, 0, s>>>(sin, t.N, 1, cnt);
    PB_LAUNCH_CHECK();
    unsigned herr = 0;
    unsigned long long hin = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaMemcpyAsync(&hin, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(err, s);
    dfree(cnt, s);
    dfree(changed, s);
    if (herr & OERR_CROSS_OWNER) {
        set_error("octree: an edge meeting the surface lies outside the all-finest region");
        return PB_ERR_ARG;
    }
    // the finest-lattice arrays are no longer needed
    dfree(g->inside, s);
    dfree(g->rowstart, s);
    g->rowstart = nullptr;
    g->inside = sin;
    g->ninside = (long long)hin;
    g->is_oct = 1;
    GridGeo fg;
    fg.nx = (int)t.N;
    fg.ny = 1;
    fg.nz = 1;
    fg.N = t.N;
    for (int d = 0; d < 3; ++d) {
        fg.o[d] = t.o[d];
        g->center[d] = t.o[d] + 0.5 * (double)t.NL * hf;
    }
    fg.h = hf;
    g->geo = fg;
    return PB_OK;
}

void oct_grid_free(pb_grid *g, cudaStream_t s) {
    OctDev &t = g->ot;
    dfree(t.lev, s);
    dfree(t.bmap, s);
    dfree(t.blow, s);
    dfree(t.bnbr, s);
    dfree(t.okind, s);
    dfree(g->cslot_b, s);
}

// ------------------------------------------------------- coefficients ---
pb_status oct_boundary_rhs(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    const OctDev &t = g->ot;
    OctSys *os = sys->os;
    const LevelConst lc = level_const(sys);
    const BcDesc bd = bc_desc(sys);
    const long long N = t.N;
    unsigned *err = (unsigned *)dalloc(sizeof(unsigned), s);
    double *tlift = (double *)dalloc(sizeof(double) * (os->ntr > 0 ? os->ntr : 1), s);
    if (!err || !tlift) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    k_oct_bc<<<cdiv(N, OT), OT, 0, s>>>(t, bd, sys->bc);
    PB_LAUNCH_CHECK();
    if (os->ntr > 0) {
        k_oct_tr_fill<<<cdiv(os->ntr, 128), 128, 0, s>>>(t, bd, g->inside, lc, sys->p.eps_out,
                                                         os->tr_slot, os->ntr, os->tr_ptr, os->tr_col,
                                                         os->tr_val, os->tr_val32, os->tr_diag,
                                                         sys->diag, tlift);
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaMemsetAsync(sys->rhs, 0, sizeof(double) * N, s));
    const double coef0 = 4.0 * M_PI * sys->lB;
    k_oct_deposit<<<cdiv(8 * g->na, 128), 128, 0, s>>>(g->atoms, g->na, g->vgeo, t, g->cells, coef0,
                                                        sys->rhs, err);
    PB_LAUNCH_CHECK();
    k_oct_lift<<<cdiv(N, OT), OT, 0, s>>>(t, bd, sys->W[0], sys->W[1], sys->W[2], sys->bc, os->tr_row,
                                          tlift, sys->rhs);
    PB_LAUNCH_CHECK();
    unsigned herr = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(err, s);
    dfree(tlift, s);
    if (herr & OERR_DEPOSIT) {
        set_error("octree: a charge cell corner is not a regular node of the finest level");
        return PB_ERR_ARG;
    }
    if (herr) {
        set_error("octree: inconsistent level-transition row (flags %u)", herr);
        return PB_ERR_ARG;
    }
    return PB_OK;
}

pb_status oct_assemble(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    const OctDev &t = g->ot;
    const long long N = t.N;
    PadGeo &p = sys->pad;
    p.nx = (int)N;
    p.ny = 1;
    p.nz = 1;
    p.sx = (int)N;
    p.sxy = N;
    p.Np = N;
    p.N = N;
    for (int d = 0; d < 3; ++d) sys->W[d] = (double *)dalloc(sizeof(double) * N, s);
    sys->diag = (double *)dalloc(sizeof(double) * N, s);
    sys->rhs = (double *)dalloc(sizeof(double) * N, s);
    sys->bc = (double *)dalloc(sizeof(double) * N, s);
    sys->phi = (double *)dalloc(sizeof(double) * N, s);
    sys->code = (uint8_t *)dalloc((size_t)((N + 15) & ~15ll), s);
    for (int d = 0; d < 3; ++d) sys->w32[d] = (float *)dalloc(sizeof(float) * N, s);
    if (!sys->W[0] || !sys->W[1] || !sys->W[2] || !sys->diag || !sys->rhs || !sys->bc || !sys->phi ||
        !sys->code || !sys->w32[0] || !sys->w32[1] || !sys->w32[2])
        return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(sys->code, 0, (size_t)((N + 15) & ~15ll), s));
    PB_CUDA_TRY(cudaMemsetAsync(sys->phi, 0, sizeof(double) * N, s));
    for (int d = 0; d < 3; ++d) PB_CUDA_TRY(cudaMemsetAsync(sys->w32[d], 0, sizeof(float) * N, s));
    const LevelConst lc = level_const(sys);
    k_oct_coef_pure<<<cdiv(N, OT), OT, 0, s>>>(t, g->inside, lc, sys->p.eps_in, sys->p.eps_out,
                                               sys->W[0], sys->W[1], sys->W[2], sys->code);
    PB_LAUNCH_CHECK();
    if (g->ncross > 0) {
        k_oct_coef_special<<<cdiv(g->ncross, OT), OT, 0, s>>>(
            g->cid, g->calpha, g->ncross, N, t.hf, sys->p.eps_in, sys->p.eps_out, sys->W[0],
            sys->W[1], sys->W[2], sys->w32[0], sys->w32[1], sys->w32[2], sys->code);
        PB_LAUNCH_CHECK();
    }
    k_oct_diag<<<cdiv(N, OT), OT, 0, s>>>(t, sys->W[0], sys->W[1], sys->W[2], g->inside, lc,
                                          sys->diag);
    PB_LAUNCH_CHECK();
    k_oct_code_kind<<<cdiv(N, OT), OT, 0, s>>>(t, sys->code);
    PB_LAUNCH_CHECK();
    // level-transition rows
    OctSys *os = new (std::nothrow) OctSys();
    if (!os) return PB_ERR_OOM;
    sys->os = os;
    long long *cnt = (long long *)dalloc(sizeof(long long), s);
    os->tr_row = (int *)dalloc(sizeof(int) * N, s);
    os->tpart = (double *)dalloc(sizeof(double) * 4, s);
    os->tcount = (unsigned *)dalloc(sizeof(unsigned), s);
    if (!cnt || !os->tr_row || !os->tpart || !os->tcount) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(long long), s));
    PB_CUDA_TRY(cudaMemsetAsync(os->tr_row, 0xff, sizeof(int) * N, s));
    PB_CUDA_TRY(cudaMemsetAsync(os->tpart, 0, sizeof(double) * 4, s));
    PB_CUDA_TRY(cudaMemsetAsync(os->tcount, 0, sizeof(unsigned), s));
    int *slots_any = (int *)dalloc(sizeof(int) * N, s);
    if (!slots_any) return PB_ERR_OOM;
    k_oct_tr_list<<<cdiv(N, OT), OT, 0, s>>>(t, cnt, slots_any);
    PB_LAUNCH_CHECK();
    long long ntr = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&ntr, cnt, sizeof(long long), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    os->ntr = ntr;
    const long long ntr1 = ntr > 0 ? ntr : 1;
    os->tr_slot = (int *)dalloc(sizeof(int) * ntr1, s);
    os->tr_ptr = (long long *)dalloc(sizeof(long long) * (ntr1 + 1), s);
    os->tr_diag = (double *)dalloc(sizeof(double) * ntr1, s);
    if (!os->tr_slot || !os->tr_ptr || !os->tr_diag) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(os->tr_ptr, 0, sizeof(long long) * (ntr1 + 1), s));
    unsigned *err = (unsigned *)dalloc(sizeof(unsigned), s);
    if (!err) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    long long nnz = 0;
    if (ntr > 0) {
        // rows in increasing slot order
        size_t tb = 0;
        PB_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, slots_any, os->tr_slot, (int)ntr, 0, 32, s));
        void *tmp = dalloc(tb, s);
        if (!tmp) return PB_ERR_OOM;
        PB_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tb, slots_any, os->tr_slot, (int)ntr, 0, 32, s));
        note_launch(2);
        dfree(tmp, s);
        k_oct_tr_rowmap<<<cdiv(ntr, OT), OT, 0, s>>>(os->tr_slot, ntr, os->tr_row);
        PB_LAUNCH_CHECK();
        long long *rn = (long long *)dalloc(sizeof(long long) * ntr, s);
        if (!rn) return PB_ERR_OOM;
        const BcDesc bd = bc_desc(sys);
        k_oct_tr_count<<<cdiv(ntr, 128), 128, 0, s>>>(t, bd, g->inside, lc, sys->p.eps_out,
                                                       os->tr_slot, ntr, rn, err);
        PB_LAUNCH_CHECK();
        tb = 0;
        PB_CUDA_TRY(cub::DeviceScan::InclusiveSum(nullptr, tb, rn, os->tr_ptr + 1, (int)ntr, s));
        tmp = dalloc(tb, s);
        if (!tmp) return PB_ERR_OOM;
        PB_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp, tb, rn, os->tr_ptr + 1, (int)ntr, s));
        note_launch(1);
        PB_CUDA_TRY(cudaMemcpyAsync(&nnz, os->tr_ptr + ntr, sizeof(long long), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        dfree(tmp, s);
        dfree(rn, s);
    }
    dfree(slots_any, s);
    dfree(cnt, s);
    unsigned herr = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(err, s);
    if (herr) {
        set_error("octree: inconsistent level-transition row (flags %u)", herr);
        return PB_ERR_ARG;
    }
    os->nnz = nnz;
    {
        unsigned long long *c = (unsigned long long *)dalloc(sizeof(unsigned long long), s);
        if (!c) return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(unsigned long long), s));
        k_count_flags<<<num_sms() * 4, OT, 0, s>>>(t.okind, N, 0, c);
        PB_LAUNCH_CHECK();
        unsigned long long h0 = 0;
        PB_CUDA_TRY(cudaMemcpyAsync(&h0, c, sizeof(h0), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        dfree(c, s);
        os->nunk = (long long)h0 + ntr;
    }
    const long long nnz1 = nnz > 0 ? nnz : 1;
    os->tr_col = (int *)dalloc(sizeof(int) * nnz1, s);
    os->tr_val = (double *)dalloc(sizeof(double) * nnz1, s);
    os->tr_val32 = (float *)dalloc(sizeof(float) * nnz1, s);
    os->npart = 2 * (int)std::max<long long>(cdiv(ntr1, OT), 1) + 8;
    os->partials = (double *)dalloc(sizeof(double) * os->npart, s);
    if (!os->tr_col || !os->tr_val || !os->tr_val32 || !os->partials) return PB_ERR_OOM;
    return oct_boundary_rhs(sys, s);
}

void oct_system_free(pb_system *sys, cudaStream_t s) {
    OctSys *os = sys->os;
    if (!os) return;
    void *ptrs[] = {os->tr_slot, os->tr_row, os->tr_ptr, os->tr_col, os->tr_val, os->tr_val32,
                    os->tr_diag, os->tpart, os->partials, os->tcount};
    for (void *p : ptrs) dfree(p, s);
    delete os;
    sys->os = nullptr;
}

pb_status oct_fill_kappa(const pb_system *sys, double *dst, cudaStream_t s) {
    const OctDev &t = sys->g->ot;
    k_oct_kappa<<<cdiv(t.N, OT), OT, 0, s>>>(t, sys->g->inside, level_const(sys), dst);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

// ------------------------------------------------------------ solver ---
namespace {

template <typename T>
OctArgs<T> oct_args(pb_system *sys) {
    OctArgs<T> A{};
    A.t = sys->g->ot;
    A.code = sys->code;
    for (int d = 0; d < 3; ++d) {
        A.w32[d] = sys->w32[d];
        A.W[d] = sys->W[d];
    }
    A.diag = sys->diag;
    A.lc = level_const(sys);
    OctSys *os = sys->os;
    A.tr_slot = os->tr_slot;
    A.tr_ptr = os->tr_ptr;
    A.tr_col = os->tr_col;
    if constexpr (sizeof(T) == 4) A.tr_val = os->tr_val32;
    else A.tr_val = os->tr_val;
    A.tr_diag = os->tr_diag;
    A.ntr = os->ntr;
    A.st = sys->st;
    A.partials = sys->partials;
    return A;
}

template <typename T>
void oct_iteration(pb_system *sys, OctArgs<T> A, T *z, T *pold, T *p, T *x, cudaStream_t s) {
    A.z = z;
    A.pold = pold;
    A.p = p;
    A.x = x;
    A.zz = z;
    k_oct_pure<T, OM_P><<<pure_grid<T, OM_P>(), OB, 0, s>>>(A);
    k_oct_pure<T, OM_U><<<pure_grid<T, OM_U>(), OB, 0, s>>>(A);
    note_launch(2);
}

pb_status oct_ensure_ws(pb_system *sys, int precision, cudaStream_t s) {
    const long long N = sys->g->ot.N;
    if (!sys->st) {
        sys->st = (CgState *)dalloc(sizeof(CgState), s);
        if (!sys->st) return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(sys->st, 0, sizeof(CgState), s));
        PB_CUDA_TRY(cudaMallocHost((void **)&sys->h_st, 4 * sizeof(CgState)));
        const int G = std::max(std::max(pure_grid<float, OM_P>(), pure_grid<float, OM_U>()),
                               std::max(pure_grid<double, OM_P>(), pure_grid<double, OM_U>()));
        sys->npartials = 2 * (int)std::max<long long>(cdiv(N, OT), G) + 64;
        sys->partials = (double *)dalloc(sizeof(double) * sys->npartials, s);
        if (!sys->partials) return PB_ERR_OOM;
    }
    const size_t b32 = sizeof(float) * (size_t)N, b64 = sizeof(double) * (size_t)N;
    if (precision == PB_MIXED && !sys->z32) {
        sys->z32 = (float *)dalloc(b32, s);
        sys->pa32 = (float *)dalloc(b32, s);
        sys->pb32 = (float *)dalloc(b32, s);
        sys->d32 = (float *)dalloc(b32, s);
        if (!sys->z32 || !sys->pa32 || !sys->pb32 || !sys->d32) return PB_ERR_OOM;
        for (float *q : {sys->z32, sys->pa32, sys->pb32, sys->d32})
            PB_CUDA_TRY(cudaMemsetAsync(q, 0, b32, s));
    }
    if (precision == PB_FP64 && !sys->z64) {
        sys->z64 = (double *)dalloc(b64, s);
        sys->pa64 = (double *)dalloc(b64, s);
        sys->pb64 = (double *)dalloc(b64, s);
        sys->x64 = (double *)dalloc(b64, s);
        if (!sys->z64 || !sys->pa64 || !sys->pb64 || !sys->x64) return PB_ERR_OOM;
        for (double *q : {sys->z64, sys->pa64, sys->pb64, sys->x64})
            PB_CUDA_TRY(cudaMemsetAsync(q, 0, b64, s));
    }
    return PB_OK;
}

pb_status oct_state(pb_system *sys, double rho, double rr0, double rr_stop, int max_iter,
                    cudaStream_t s, int profile = 0) {
    CgState h{};
    h.profile = profile;
    h.rho = rho;
    h.rr0 = rr0;
    h.rr = rr0;
    h.rr_stop = rr_stop;
    h.max_iter = max_iter;
    CgState *stage = sys->h_st + 2;
    *stage = h;
    PB_CUDA_TRY(cudaMemcpyAsync(sys->st, stage, sizeof(CgState), cudaMemcpyHostToDevice, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return PB_OK;
}

pb_status oct_sync(pb_system *sys, cudaStream_t s) {
    PB_CUDA_TRY(cudaMemcpyAsync(sys->h_st, sys->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return PB_OK;
}

pb_status oct_residual(pb_system *sys, bool fp32_out, cudaStream_t s) {
    const OctDev &t = sys->g->ot;
    OctSys *os = sys->os;
    if (fp32_out)
        k_oct_residual<float><<<cdiv(t.N, OT), OT, 0, s>>>(
            t, sys->phi, sys->rhs, sys->W[0], sys->W[1], sys->W[2], sys->diag, os->tr_row,
            os->tr_ptr, os->tr_col, os->tr_val, sys->z32, sys->st, sys->partials);
    else
        k_oct_residual<double><<<cdiv(t.N, OT), OT, 0, s>>>(
            t, sys->phi, sys->rhs, sys->W[0], sys->W[1], sys->W[2], sys->diag, os->tr_row,
            os->tr_ptr, os->tr_col, os->tr_val, sys->z64, sys->st, sys->partials);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

// iterations until the device state says done (two chunks in flight)
template <typename T>
pb_status oct_run(pb_system *sys, T *z, T *pa, T *pb, T *x, double deadline, cudaStream_t s,
                  int *iters) {
    OctArgs<T> A = oct_args<T>(sys);
    T *bufs[2] = {pa, pb};
    int cur = 0;
    const int chunk = 16;
    cudaEvent_t ev[2];
    PB_CUDA_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    PB_CUDA_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    CgState *hs = sys->h_st;
    pb_status rc = PB_OK;
    auto issue = [&](int slot) -> pb_status {
        for (int c = 0; c < chunk; ++c) {
            oct_iteration<T>(sys, A, z, bufs[cur], bufs[cur ^ 1], x, s);
            cur ^= 1;
        }
        PB_CUDA_TRY(cudaGetLastError());
        PB_CUDA_TRY(cudaMemcpyAsync(hs + slot, sys->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaEventRecord(ev[slot], s));
        return PB_OK;
    };
    const long long max_chunks = (long long)hs[2].max_iter / chunk + 4;
    long long issued = 2;
    int slot = 0;
    if ((rc = issue(0)) == PB_OK) rc = issue(1);
    while (rc == PB_OK) {
        cudaError_t e = cudaEventSynchronize(ev[slot]);
        if (e != cudaSuccess) {
            set_error("octree PCG chunk failed: %s", cudaGetErrorString(e));
            rc = PB_ERR_CUDA;
            break;
        }
        if (hs[slot].done) break;
        if (deadline > 0.0 && wall_s() > deadline) {
            rc = PB_ERR_TIMEOUT;
            break;
        }
        if (++issued > max_chunks) {
            set_error("octree PCG state stopped advancing");
            rc = PB_ERR_CUDA;
            break;
        }
        rc = issue(slot);
        slot ^= 1;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("octree PCG failed: %s", cudaGetErrorString(e));
        rc = PB_ERR_CUDA;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc == PB_OK) {
        if ((rc = oct_sync(sys, s)) != PB_OK) return rc;
        *iters = hs[0].iter;
    }
    return rc;
}

}  // namespace

pb_status oct_solve(pb_system *sys, const pb_solve_opts *o, cudaStream_t s, pb_solve_stats *stats) {
    const double t_start = wall_s();
    const double deadline = o->time_budget_s > 0.0 ? t_start + o->time_budget_s : 0.0;
    const OctDev &t = sys->g->ot;
    const long long N = t.N;
    pb_status rc = oct_ensure_ws(sys, o->precision, s);
    if (rc != PB_OK) return rc;
    const int max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    const int max_outer = o->max_outer > 0 ? o->max_outer : 30;
    const double rtol = o->rtol > 0.0 ? o->rtol : 1e-8;
    const double inner_rtol = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-6;
    const BcDesc bd = bc_desc(sys);
    PB_CUDA_TRY(cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    int iters = 0, outer = 0, status = PB_OK;
    double fn2 = 0.0, res2 = 0.0;
    const unsigned nb = cdiv(N, OT);
    if (o->precision == PB_MIXED) {
        if ((rc = oct_residual(sys, true, s)) != PB_OK) return rc;
        if ((rc = oct_sync(sys, s)) != PB_OK) return rc;
        fn2 = res2 = sys->h_st->res64;
        outer = 1;
        int stagnant = 0;
        while (fn2 > 0.0 && res2 > rtol * rtol * fn2) {
            if (outer > max_outer || iters >= max_iter) {
                status = PB_ERR_NOCONV;
                break;
            }
            const double rel = sqrt(res2 / fn2);
            double itol = std::max(inner_rtol, 0.5 * rtol / rel);
            if (itol > 0.5) itol = 0.5;
            if ((rc = oct_state(sys, sys->h_st->rz64, res2, itol * itol * res2, max_iter - iters, s)) != PB_OK)
                return rc;
            PB_CUDA_TRY(cudaMemsetAsync(sys->d32, 0, sizeof(float) * N, s));
            PB_CUDA_TRY(cudaMemsetAsync(sys->pa32, 0, sizeof(float) * N, s));
            int it = 0;
            rc = oct_run<float>(sys, sys->z32, sys->pa32, sys->pb32, sys->d32, deadline, s, &it);
            if (rc == PB_ERR_TIMEOUT) status = PB_ERR_TIMEOUT;
            else if (rc != PB_OK) return rc;
            if (rc == PB_OK) iters += it;
            k_oct_promote<float><<<nb, OT, 0, s>>>(t, sys->phi, sys->d32);
            PB_LAUNCH_CHECK();
            if ((rc = oct_residual(sys, true, s)) != PB_OK) return rc;
            if ((rc = oct_sync(sys, s)) != PB_OK) return rc;
            const double prev = res2;
            res2 = sys->h_st->res64;
            ++outer;
            if (status == PB_ERR_TIMEOUT) break;
            if (res2 > 0.25 * prev) {
                if (++stagnant >= 3) {
                    status = PB_ERR_NOCONV;
                    break;
                }
            } else {
                stagnant = 0;
            }
        }
    } else {
        PB_CUDA_TRY(cudaMemsetAsync(sys->x64, 0, sizeof(double) * N, s));
        if ((rc = oct_residual(sys, false, s)) != PB_OK) return rc;
        if ((rc = oct_sync(sys, s)) != PB_OK) return rc;
        fn2 = res2 = sys->h_st->res64;
        outer = 1;
        while (fn2 > 0.0 && res2 > rtol * rtol * fn2) {
            if (outer > max_outer || iters >= max_iter) {
                status = PB_ERR_NOCONV;
                break;
            }
            if ((rc = oct_state(sys, sys->h_st->rz64, res2, rtol * rtol * fn2 * 0.25, max_iter - iters, s)) !=
                PB_OK)
                return rc;
            PB_CUDA_TRY(cudaMemsetAsync(sys->pa64, 0, sizeof(double) * N, s));
            int it = 0;
            rc = oct_run<double>(sys, sys->z64, sys->pa64, sys->pb64, sys->x64, deadline, s, &it);
            if (rc == PB_ERR_TIMEOUT) status = PB_ERR_TIMEOUT;
            else if (rc != PB_OK) return rc;
            if (rc == PB_OK) iters += it;
            PB_CUDA_TRY(cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            k_oct_promote<double><<<nb, OT, 0, s>>>(t, sys->phi, sys->x64);
            PB_LAUNCH_CHECK();
            if ((rc = oct_residual(sys, false, s)) != PB_OK) return rc;
            if ((rc = oct_sync(sys, s)) != PB_OK) return rc;
            res2 = sys->h_st->res64;
            ++outer;
            if (status == PB_ERR_TIMEOUT) break;
        }
    }
    k_oct_hang<<<nb, OT, 0, s>>>(t, bd, sys->phi);
    PB_LAUNCH_CHECK();
    sys->fnorm2 = fn2;
    sys->solved = 1;
    if (stats) {
        stats->status = status;
        stats->iters_inner = iters;
        stats->iters_outer = outer;
        stats->kc = 0;
        stats->true_rel_res = fn2 > 0.0 ? sqrt(res2 / fn2) : 0.0;
        stats->seconds = wall_s() - t_start;
        const long long dof = sys->os->nunk;
        stats->dof = dof;
        const long long per = o->precision == PB_MIXED ? (8 * 4 + 2) : (8 * 8 + 6 * 8 + 2);
        stats->model_bytes = (long long)iters * dof * per + (long long)outer * N * 64;
    }
    return (pb_status)status;
}

pb_status oct_apply(pb_system *sys, int precision, const void *x, void *y, cudaStream_t s) {
    const OctDev &t = sys->g->ot;
    if (!sys->st) {
        pb_status rc = oct_ensure_ws(sys, precision, s);
        if (rc != PB_OK) return rc;
    }
    if (precision == PB_MIXED) {
        OctArgs<float> A = oct_args<float>(sys);
        A.xin = (const float *)x;
        A.y = (float *)y;
        k_oct_pure<float, OM_A><<<pure_grid<float, OM_A>(), OB, 0, s>>>(A);
        PB_LAUNCH_CHECK();
    } else {
        OctArgs<double> A = oct_args<double>(sys);
        A.xin = (const double *)x;
        A.y = (double *)y;
        k_oct_pure<double, OM_A><<<pure_grid<double, OM_A>(), OB, 0, s>>>(A);
        PB_LAUNCH_CHECK();
    }
    (void)t;
    return PB_OK;
}

pb_status oct_profile(pb_system *sys, int precision, int which, int reps, cudaStream_t s) {
    pb_status rc = oct_state(sys, 1.0, 1.0, -1.0, 1 << 30, s, 1);
    if (rc != PB_OK) return rc;
    for (int r = 0; r < reps; ++r) {
        if (precision == PB_MIXED) {
            OctArgs<float> A = oct_args<float>(sys);
            A.z = A.zz = sys->z32;
            A.pold = (r & 1) ? sys->pb32 : sys->pa32;
            A.p = (r & 1) ? sys->pa32 : sys->pb32;
            A.x = sys->d32;
            if (which == 0 || which == 2) k_oct_pure<float, OM_P><<<pure_grid<float, OM_P>(), OB, 0, s>>>(A);
            if (which == 1 || which == 2) k_oct_pure<float, OM_U><<<pure_grid<float, OM_U>(), OB, 0, s>>>(A);
        } else {
            OctArgs<double> A = oct_args<double>(sys);
            A.z = A.zz = sys->z64;
            A.pold = (r & 1) ? sys->pb64 : sys->pa64;
            A.p = (r & 1) ? sys->pa64 : sys->pb64;
            A.x = sys->x64;
            if (which == 0 || which == 2) k_oct_pure<double, OM_P><<<pure_grid<double, OM_P>(), OB, 0, s>>>(A);
            if (which == 1 || which == 2) k_oct_pure<double, OM_U><<<pure_grid<double, OM_U>(), OB, 0, s>>>(A);
        }
        PB_LAUNCH_CHECK();
    }
    return PB_OK;
}

pb_status oct_energy(pb_system *sys, cudaStream_t s, pb_energy_terms *out) {
    pb_grid *g = sys->g;
    const int nb = (int)std::min<long long>(cdiv(g->ncross > 0 ? g->ncross : 1, EN_T),
                                            (long long)num_sms() * 8);
    double *partials = (double *)dalloc(sizeof(double) * 4 * nb, s);
    if (!partials) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(&sys->eacc->counter, 0, sizeof(unsigned), s));
    k_oct_energy<<<nb, EN_T, 0, s>>>(g->cid, g->cslot_b, g->calpha, g->csign, g->ncross, g->ot.N,
                                     sys->W[0], sys->W[1], sys->W[2], sys->phi, sys->Phi, sys->Psi,
                                     g->mc_w, sys->PsiN,
                                     g->ot.hf, sys->p.eps_in, sys->p.eps_out, sys->lB, partials,
                                     sys->eacc);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(sys->h_energy, &sys->eacc->out, sizeof(pb_energy_terms),
                                cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    dfree(partials, s);
    *out = *sys->h_energy;
    return PB_OK;
}

}  // namespace pbg

// ------------------------------------------------ serving-engine hooks ---
// The continuous-batching engine runs octree systems beside its launch
// table: these queue one system's pieces on the engine's stream (the
// system's CG state pointer is the engine slot's).
namespace pbg {

pb_status oct_engine_prepare(pb_system *sys, cudaStream_t s) { return oct_ensure_ws(sys, PB_MIXED, s); }

pb_status oct_engine_residual(pb_system *sys, cudaStream_t s) { return oct_residual(sys, true, s); }

// promotion of the FP32 correction and the hanging values of phi
pb_status oct_engine_promote(pb_system *sys, cudaStream_t s) {
    const OctDev &t = sys->g->ot;
    k_oct_promote<float><<<cdiv(t.N, OT), OT, 0, s>>>(t, sys->phi, sys->d32);
    PB_LAUNCH_CHECK();
    k_oct_hang<<<cdiv(t.N, OT), OT, 0, s>>>(t, bc_desc(sys), sys->phi);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

// n (even) FP32 PCG iterations starting from direction parity 0; the
// kernels do nothing once the state says done
pb_status oct_engine_iterations(pb_system *sys, int n, cudaStream_t s) {
    OctArgs<float> A = oct_args<float>(sys);
    float *bufs[2] = {sys->pa32, sys->pb32};
    for (int c = 0; c < n; ++c) oct_iteration<float>(sys, A, sys->z32, bufs[c & 1], bufs[(c & 1) ^ 1], sys->d32, s);
    PB_CUDA_TRY(cudaGetLastError());
    return PB_OK;
}

}  // namespace pbg
