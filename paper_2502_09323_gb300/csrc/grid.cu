// Grid placement, node classification and the surface-crossing edge list.
//
// Compiled with --fmad=false: every FP64 expression here is evaluated as
// written (no fused multiply-add), so node positions, inside tests and
// inside fractions are reproducible to the bit on any IEEE-754 machine.
//
// Sec. 2.1: eps(r) = eps_m in the solute (union of atom balls), eps_s outside.
// Sec. 3.2: an edge that meets the molecular surface gets the weighted harmonic
//   average permittivity of Eq. WHA, whose weight alpha is the fraction of the
//   edge inside the solute; the point where the surface cuts the edge is where
//   Sec. 3.3.1 concentrates the polarisation charge of that edge.
// Sec. 2.3 / 3.4: the box is a cube of side fill * molecular extent (perfil).
#include <math.h>

#include <cmath>
#include <cub/block/block_reduce.cuh>
#include <cub/block/block_scan.cuh>

#include "pb_internal.h"

namespace pbg {

namespace {

constexpr int PREP_THREADS = 1024;
constexpr int CHUNK_THREADS = 256;
constexpr int CHUNK_BYTES = CHUNK_THREADS * 16;

struct OrOp {
    __device__ __forceinline__ unsigned operator()(unsigned a, unsigned b) const { return a | b; }
};
struct MinOp {
    __device__ __forceinline__ double operator()(double a, double b) const { return fmin(a, b); }
};
struct MaxOp {
    __device__ __forceinline__ double operator()(double a, double b) const { return fmax(a, b); }
};

__device__ __forceinline__ double node_coord(const GridGeo &g, int d, long long i) {
    return g.o[d] + (double)i * g.h;
}

__device__ __forceinline__ long long clampll(long long v, long long lo, long long hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// ----------------------------------------------------------- atom layout --
__global__ void k_aos_to_soa(const double *__restrict__ aos, double *__restrict__ soa,
                             long long na) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= na) return;
#pragma unroll
    for (int d = 0; d < 5; ++d) soa[d * na + i] = aos[5 * i + d];
}

// ------------------------------------------------- validation + placement --
// One block: checks the atoms, reduces the bounding box of the balls and,
// when asked, places the grid (cube of side fill*extent centred on the box).
// Then checks that every charge's trilinear cell has interior corners only.
__global__ void __launch_bounds__(PREP_THREADS)
k_prep(const double *__restrict__ atoms, long long na, int auto_place, int nmax,
       double fill, int n0, int n1, int n2, double ox, double oy, double oz,
       double hgiven, BuildInfo *info) {
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *R = atoms + 3 * na,
                 *Q = atoms + 4 * na;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double rmax = 0.0;
    unsigned err = 0;
    for (long long i = threadIdx.x; i < na; i += blockDim.x) {
        double c[3] = {X[i], Y[i], Z[i]};
        double r = R[i], q = Q[i];
        if (!isfinite(c[0]) || !isfinite(c[1]) || !isfinite(c[2]) || !isfinite(q) ||
            !isfinite(r) || !(r > 0.0))
            err |= ERRF_ATOM_VALUE;
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], c[d] - r);
            hi[d] = fmax(hi[d], c[d] + r);
        }
        rmax = fmax(rmax, r);
    }
    using BR = cub::BlockReduce<double, PREP_THREADS>;
    using BRU = cub::BlockReduce<unsigned, PREP_THREADS>;
    __shared__ typename BR::TempStorage tmp;
    __shared__ typename BRU::TempStorage tmpu;
    __shared__ double s_lo[3], s_hi[3], s_rmax, s_o[3], s_h;
    for (int d = 0; d < 3; ++d) {
        double v = BR(tmp).Reduce(lo[d], MinOp());
        __syncthreads();
        if (threadIdx.x == 0) s_lo[d] = v;
        v = BR(tmp).Reduce(hi[d], MaxOp());
        __syncthreads();
        if (threadIdx.x == 0) s_hi[d] = v;
    }
    double rm = BR(tmp).Reduce(rmax, MaxOp());
    __syncthreads();
    unsigned eb = BRU(tmpu).Reduce(err, OrOp());
    if (threadIdx.x == 0) {
        s_rmax = rm;
        if (auto_place) {
            double ext = 0.0;
            for (int d = 0; d < 3; ++d)
                if (s_hi[d] - s_lo[d] > ext) ext = s_hi[d] - s_lo[d];
            double L = fill * ext;
            s_h = L / (double)(nmax - 1);
            for (int d = 0; d < 3; ++d) s_o[d] = 0.5 * (s_lo[d] + s_hi[d]) - 0.5 * L;
        } else {
            s_h = hgiven;
            s_o[0] = ox;
            s_o[1] = oy;
            s_o[2] = oz;
        }
        for (int d = 0; d < 3; ++d) {
            info->lo[d] = s_lo[d];
            info->hi[d] = s_hi[d];
            info->origin[d] = s_o[d];
        }
        info->h = s_h;
        info->rmax = s_rmax;
        info->err = eb;
    }
    __syncthreads();
    // trilinear cell of each charge: clamp(floor((x - o)/h), 0, n-2); all
    // eight corners must be interior unknowns
    int nn[3] = {n0, n1, n2};
    unsigned cerr = 0;
    for (long long i = threadIdx.x; i < na; i += blockDim.x) {
        double c[3] = {X[i], Y[i], Z[i]};
        for (int d = 0; d < 3; ++d) {
            double u = (c[d] - s_o[d]) / s_h;
            double fl = floor(u);
            long long ci;
            if (!(fl == fl)) ci = -1;
            else if (fl < -1e18) ci = -1;
            else if (fl > 1e18) ci = nn[d];
            else ci = clampll((long long)fl, 0, nn[d] - 2);
            if (ci < 1 || ci + 1 > nn[d] - 2) cerr |= ERRF_CHARGE_CELL;
        }
    }
    unsigned ce = BRU(tmpu).Reduce(cerr, OrOp());
    if (threadIdx.x == 0) info->err |= ce;
}

// --------------------------------------------------------- classification --
// Node a is inside when (dx*dx + dy*dy) + dz*dz < R*R for some atom.  One
// block per atom over the z-columns of the ball's bounding box (one node of
// margin on each side): a column keeps its dx*dx + dy*dy, and one whose
// value already reaches R*R holds no inside node (adding dz*dz >= 0 cannot
// lower it).
__global__ void k_classify(const double *__restrict__ atoms, long long na, GridGeo g,
                           uint8_t *__restrict__ inside) {
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *R = atoms + 3 * na;
    int nn[3] = {g.nx, g.ny, g.nz};
    for (long long at = blockIdx.x; at < na; at += gridDim.x) {
        double c[3] = {X[at], Y[at], Z[at]};
        double r = R[at];
        long long lo[3], hi[3], ext[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = clampll((long long)floor((c[d] - r - g.o[d]) / g.h) - 1, 0, nn[d] - 1);
            hi[d] = clampll((long long)ceil((c[d] + r - g.o[d]) / g.h) + 1, 0, nn[d] - 1);
            ext[d] = hi[d] - lo[d] + 1;
        }
        const double R2 = r * r;
        const long long cols = ext[0] * ext[1];
        for (long long t = threadIdx.x; t < cols; t += blockDim.x) {
            const long long i = lo[0] + t % ext[0];
            const long long j = lo[1] + t / ext[0];
            const double dx = node_coord(g, 0, i) - c[0];
            const double dy = node_coord(g, 1, j) - c[1];
            const double q = dx * dx + dy * dy;
            if (!(q < R2)) continue;
            for (long long k = lo[2]; k <= hi[2]; ++k) {
                const double dz = node_coord(g, 2, k) - c[2];
                if (q + dz * dz < R2) inside[(k * g.ny + j) * g.nx + i] = 1;
            }
        }
    }
}

// --------------------------------------------------------------- cell list --
__device__ __forceinline__ int cell_coord(const CellList &cl, int d, double x) {
    double u = floor((x - cl.lo[d]) / cl.cs);
    if (!(u >= 0.0)) return -1;
    if (u >= (double)cl.dim[d]) return cl.dim[d];
    return (int)u;
}

__global__ void k_cell_count(const double *__restrict__ atoms, long long na, CellList cl,
                             int *__restrict__ acell, int *__restrict__ count, BuildInfo *info) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= na) return;
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = cell_coord(cl, d, atoms[d * na + i]);
    for (int d = 0; d < 3; ++d)
        if (c[d] < 0 || c[d] >= cl.dim[d]) {
            atomicOr(&info->err, ERRF_CELL_OVERFLOW);
            acell[i] = -1;
            return;
        }
    int id = (c[2] * cl.dim[1] + c[1]) * cl.dim[0] + c[0];
    acell[i] = id;
    atomicAdd(&count[id], 1);
}

// exclusive scan of count[0..n) into start[0..n], single block
template <int T>
__global__ void __launch_bounds__(T) k_scan_int(const int *__restrict__ count, int *__restrict__ start, int n) {
    using BS = cub::BlockScan<int, T>;
    __shared__ typename BS::TempStorage tmp;
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += T) {
        int i = base + threadIdx.x;
        int v = i < n ? count[i] : 0;
        int ex, agg;
        BS(tmp).ExclusiveSum(v, ex, agg);
        if (i < n) start[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += agg;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void k_cell_fill(const int *__restrict__ acell, long long na, const int *__restrict__ start,
                            int *__restrict__ cursor, int *__restrict__ list) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= na) return;
    int c = acell[i];
    if (c < 0) return;
    int pos = atomicAdd(&cursor[c], 1);
    list[start[c] + pos] = (int)i;
}

// atoms of each cell in increasing id order (the fill above is unordered)
__global__ void k_cell_sort(const int *__restrict__ start, int *__restrict__ list, int ncell) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int s = start[c], e = start[c + 1];
    for (int a = s + 1; a < e; ++a) {
        int v = list[a];
        int b = a - 1;
        while (b >= s && list[b] > v) {
            list[b + 1] = list[b];
            --b;
        }
        list[b + 1] = v;
    }
}

// ------------------------------------------------------- inside fraction --
// Interval of the edge (x_a, x_a + h e_d) inside one ball, parameter t in
// [0,1]: (u_d + t h)^2 = R^2 - |u_perp|^2 with u = x_a - c.  Split in the part
// that depends on the lattice line only (w = sqrt(R^2 - |u_perp|^2); false
// when the line misses the ball) and the part for one edge of that line.
__device__ __forceinline__ bool line_cut(const double xa[3], int d, double ce, double cf,
                                         double R, double &w) {
    const int e = (d == 0) ? 1 : 0;
    const int f = (d == 2) ? 1 : 2;
    double ue = xa[e] - ce;
    double uf = xa[f] - cf;
    double s = R * R - (ue * ue + uf * uf);
    if (!(s > 0.0)) return false;
    w = sqrt(s);
    return true;
}

// a0 = (-u_d - w)/h and a1 = (-u_d + w)/h clamped to [0,1]; false when the
// clamped interval is empty.  A division is skipped where the numerator
// already decides its clamped value (division by h > 0 is monotone and
// exact at h): n0 >= h gives a0 >= 1 and n1 <= 0 gives a1 <= 0 (empty),
// n0 <= 0 gives t0 = 0 and n1 >= h gives t1 = 1.  (A clamped -0 becomes +0,
// which changes no comparison and no union length.)
__device__ __forceinline__ bool edge_cut(double xad, double cd, double w, double h, double &t0,
                                         double &t1) {
    double ud = xad - cd;
    double n0 = -ud - w;
    double n1 = -ud + w;
    if (n0 >= h || n1 <= 0.0) return false;
    double a0 = n0 > 0.0 ? n0 / h : 0.0;
    double a1 = n1 < h ? n1 / h : 1.0;
    if (!(a1 > a0)) return false;
    t0 = a0;
    t1 = a1;
    return true;
}

// Measure of the union of the intervals of all balls meeting the edge; the
// intervals are ordered by (t0, t1) and merged.  Returns false on overflow.
// With COVER_EXIT the scan stops at the first ball whose interval is all of
// [0, 1] (alpha = 1 exactly: the merged run then starts at 0 and ends at 1).
template <bool COVER_EXIT>
__device__ bool edge_alpha(const double *__restrict__ atoms, long long na, const CellList &cl,
                           const int *__restrict__ cstart, const int *__restrict__ clist,
                           const double xa[3], int d, double h, double &alpha) {
    double t0s[MAX_EDGE_BALLS], t1s[MAX_EDGE_BALLS];
    int m = 0;
    int cc[3];
    for (int q = 0; q < 3; ++q) {
        double u = floor((xa[q] - cl.lo[q]) / cl.cs);
        cc[q] = (u < -4.0) ? -4 : ((u > (double)cl.dim[q] + 4.0) ? cl.dim[q] + 4 : (int)u);
    }
    const int e = (d == 0) ? 1 : 0;
    const int f = (d == 2) ? 1 : 2;
    const double *Ce = atoms + (long long)e * na, *Cf = atoms + (long long)f * na;
    const double *Cd = atoms + (long long)d * na, *R = atoms + 3 * na;
    for (int cz = cc[2] - 1; cz <= cc[2] + 1; ++cz) {
        if (cz < 0 || cz >= cl.dim[2]) continue;
        for (int cy = cc[1] - 1; cy <= cc[1] + 1; ++cy) {
            if (cy < 0 || cy >= cl.dim[1]) continue;
            for (int cx = cc[0] - 1; cx <= cc[0] + 1; ++cx) {
                if (cx < 0 || cx >= cl.dim[0]) continue;
                int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
                for (int s = cstart[cid]; s < cstart[cid + 1]; ++s) {
                    int at = clist[s];
                    double w, t0, t1;
                    if (!line_cut(xa, d, Ce[at], Cf[at], R[at], w)) continue;
                    if (!edge_cut(xa[d], Cd[at], w, h, t0, t1)) continue;
                    if (COVER_EXIT && !(t0 > 0.0) && !(t1 < 1.0)) {
                        alpha = 1.0;
                        return true;
                    }
                    if (m == MAX_EDGE_BALLS) return false;
                    // insertion by (t0, t1)
                    int b = m - 1;
                    while (b >= 0 && (t0s[b] > t0 || (t0s[b] == t0 && t1s[b] > t1))) {
                        t0s[b + 1] = t0s[b];
                        t1s[b + 1] = t1s[b];
                        --b;
                    }
                    t0s[b + 1] = t0;
                    t1s[b + 1] = t1;
                    ++m;
                }
            }
        }
    }
    if (m == 0) {
        alpha = 0.0;
        return true;
    }
    double total = 0.0, c0 = t0s[0], c1 = t1s[0];
    for (int q = 1; q < m; ++q) {
        if (t0s[q] <= c1) {
            if (t1s[q] > c1) c1 = t1s[q];
        } else {
            total += c1 - c0;
            c0 = t0s[q];
            c1 = t1s[q];
        }
    }
    total += c1 - c0;
    alpha = total;
    return true;
}

struct EdgeRef {
    int d;
    long long a, b;
    long long ijk[3];
};

__device__ __forceinline__ EdgeRef edge_ref(const GridGeo &g, long long e) {
    EdgeRef r;
    r.d = (int)(e / g.N);
    r.a = e - (long long)r.d * g.N;
    r.ijk[0] = r.a % g.nx;
    r.ijk[1] = (r.a / g.nx) % g.ny;
    r.ijk[2] = r.a / ((long long)g.nx * g.ny);
    long long stride = r.d == 0 ? 1 : (r.d == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
    r.b = r.a + stride;
    return r;
}

// Candidate edges.  An edge's inside fraction can lie strictly between 0 and
// 1 only when some ball's interval on it is partial (t0 > 0 or t1 < 1): on
// every other edge each interval is empty or all of [0, 1], so alpha is 0 or
// 1 and the edge is listed exactly when its end nodes differ in `inside`.
// One block per atom, one thread per lattice line (direction d and the node
// indices of the two other axes) through the ball's bounding box.  Along a
// line both a0 and a1 of edge_cut fall as the edge moves up (x_a[d]
// enters through u_d = x_a[d] - c[d] and every rounded step after it is
// monotone), so the scan going up stops at the first edge with t0 = 0 and the
// scan coming down at the first with t1 = 1: every edge between the two has
// the interval [0, 1].  Candidates get flag byte 2, and the edges whose
// interval for this ball is all of [0, 1] get cov byte 1: on those the union
// is [0, 1] whatever the other balls add, so alpha = 1 exactly.  (Several
// balls may write the same byte, always with the same value.)
__global__ void k_edge_cand(const double *__restrict__ atoms, long long na, GridGeo g,
                            uint8_t *__restrict__ flags, uint8_t *__restrict__ cov) {
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *R = atoms + 3 * na;
    const int nn[3] = {g.nx, g.ny, g.nz};
    const long long step[3] = {1, (long long)g.nx, (long long)g.nx * g.ny};
    for (long long at = blockIdx.x; at < na; at += gridDim.x) {
        const double c[3] = {X[at], Y[at], Z[at]};
        const double r = R[at];
        long long lo[3], hi[3], ext[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = clampll((long long)floor((c[d] - r - g.o[d]) / g.h) - 1, 0, nn[d] - 1);
            hi[d] = clampll((long long)ceil((c[d] + r - g.o[d]) / g.h) + 1, 0, nn[d] - 1);
            ext[d] = hi[d] - lo[d] + 1;
        }
        const long long nl0 = ext[1] * ext[2], nl1 = ext[0] * ext[2], nl2 = ext[0] * ext[1];
        for (long long t = threadIdx.x; t < nl0 + nl1 + nl2; t += blockDim.x) {
            int d;
            long long q;
            if (t < nl0) {
                d = 0;
                q = t;
            } else if (t < nl0 + nl1) {
                d = 1;
                q = t - nl0;
            } else {
                d = 2;
                q = t - nl0 - nl1;
            }
            const int e = (d == 0) ? 1 : 0;
            const int f = (d == 2) ? 1 : 2;
            const long long ie = lo[e] + q % ext[e];
            const long long jf = lo[f] + q / ext[e];
            const long long ilo = lo[d];
            const long long ihi = hi[d] < (long long)nn[d] - 2 ? hi[d] : (long long)nn[d] - 2;
            if (ihi < ilo) continue;
            double xa[3];
            xa[d] = 0.0;
            xa[e] = node_coord(g, e, ie);
            xa[f] = node_coord(g, f, jf);
            double w;
            if (!line_cut(xa, d, c[e], c[f], r, w)) continue;
            const long long base = (long long)d * g.N + ie * step[e] + jf * step[f];
            long long iu = ihi + 1, id = ihi + 1;
            bool cov_iu = false;
            for (long long i = ilo; i <= ihi; ++i) {
                double t0, t1;
                if (!edge_cut(node_coord(g, d, i), c[d], w, g.h, t0, t1)) continue;
                if (t0 > 0.0 || t1 < 1.0) flags[base + i * step[d]] = 2;
                if (!(t0 > 0.0)) {
                    iu = i;
                    cov_iu = !(t1 < 1.0);
                    break;
                }
            }
            for (long long i = ihi; i > iu; --i) {
                double t0, t1;
                if (!edge_cut(node_coord(g, d, i), c[d], w, g.h, t0, t1)) continue;
                if (t0 > 0.0 || t1 < 1.0) flags[base + i * step[d]] = 2;
                if (!(t1 < 1.0)) {
                    id = i;
                    break;
                }
            }
            // covered: iu when its t1 is 1, and every edge from iu + 1 to id
            if (cov_iu) cov[base + iu * step[d]] = 1;
            if (id <= ihi)
                for (long long i = iu + 1; i <= id; ++i) cov[base + i * step[d]] = 1;
        }
    }
}

// flag[e] = 1 when edge e is listed: 0 < alpha < 1 or its end nodes differ in
// `inside`.  One block per 4096 edges.  Edges whose end nodes differ are
// listed; the others are listed only if they are candidates not covered by
// one ball, and for those the block computes the inside fraction (union of
// all balls' intervals): they are gathered in shared memory and shared out
// over the block.
__global__ void __launch_bounds__(CHUNK_THREADS)
k_edge_flags(const double *__restrict__ atoms, long long na, GridGeo g, CellList cl,
             const int *__restrict__ cstart, const int *__restrict__ clist,
             const uint8_t *__restrict__ inside, uint8_t *__restrict__ flags,
             const uint8_t *__restrict__ cov, BuildInfo *info) {
    __shared__ uint4 s_fl[CHUNK_THREADS];
    __shared__ int s_list[CHUNK_BYTES];
    __shared__ int s_list_n;
    if (threadIdx.x == 0) s_list_n = 0;
    __syncthreads();
    const long long tile = (long long)blockIdx.x * CHUNK_BYTES;
    uint4 v = reinterpret_cast<const uint4 *>(flags)[(long long)blockIdx.x * CHUNK_THREADS +
                                                     threadIdx.x];
    unsigned w[4] = {v.x, v.y, v.z, v.w};
    uint4 cv = make_uint4(0u, 0u, 0u, 0u);
    if (v.x | v.y | v.z | v.w)
        cv = reinterpret_cast<const uint4 *>(cov)[(long long)blockIdx.x * CHUNK_THREADS +
                                                 threadIdx.x];
    const unsigned cw[4] = {cv.x, cv.y, cv.z, cv.w};
    // first edge of this thread's 16, then stepped node by node
    long long e0 = tile + 16ll * threadIdx.x;
    int d = (int)(e0 / g.N);
    long long a = e0 - (long long)d * g.N;
    long long i = a % g.nx, row = a / g.nx;
    long long j = row % g.ny, k = row / g.ny;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned out = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            unsigned u = (w[q] >> (8 * b)) & 0xffu;
            unsigned fl = 0;
            if (d < 3) {
                long long id = d == 0 ? i : (d == 1 ? j : k);
                long long nd = d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
                long long st = d == 0 ? 1 : (d == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
                const bool differ = id < nd - 1 && inside[a] != inside[a + st];
                const bool covered = ((cw[q] >> (8 * b)) & 0xffu) != 0u;
                if (u == 2u && !differ && !covered) {
                    int p = atomicAdd(&s_list_n, 1);
                    s_list[p] = 16 * threadIdx.x + 4 * q + b;
                } else if (differ) {
                    fl = 1;
                }
            }
            out |= fl << (8 * b);
            ++a;
            if (++i == g.nx) {
                i = 0;
                if (++j == g.ny) {
                    j = 0;
                    if (++k == g.nz) {
                        k = 0;
                        a = 0;
                        ++d;
                    }
                }
            }
        }
        w[q] = out;
    }
    s_fl[threadIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
    __syncthreads();
    uint8_t *sb = reinterpret_cast<uint8_t *>(s_fl);
    const int n = s_list_n;
    for (int p = threadIdx.x; p < n; p += CHUNK_THREADS) {
        const int off = s_list[p];
        EdgeRef r = edge_ref(g, tile + off);
        double xa[3] = {node_coord(g, 0, r.ijk[0]), node_coord(g, 1, r.ijk[1]),
                        node_coord(g, 2, r.ijk[2])};
        // an edge met by too many balls is listed, so that the record pass,
        // which reports the overflow, meets it again
        double al;
        if (!edge_alpha<true>(atoms, na, cl, cstart, clist, xa, r.d, g.h, al)) al = 0.5;
        sb[off] = (al > 0.0 && al < 1.0) ? 1 : 0;
    }
    __syncthreads();
    reinterpret_cast<uint4 *>(flags)[(long long)blockIdx.x * CHUNK_THREADS + threadIdx.x] =
        s_fl[threadIdx.x];
}

// ------------------------------------------------- ordered compaction --
__device__ __forceinline__ int nz_bytes(uint4 v) {
    unsigned w[4] = {v.x, v.y, v.z, v.w};
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = 0; b < 4; ++b) c += ((w[q] >> (8 * b)) & 0xffu) != 0u;
    return c;
}

__global__ void __launch_bounds__(CHUNK_THREADS)
k_chunk_count(const uint4 *__restrict__ flags, int *__restrict__ counts) {
    using BR = cub::BlockReduce<int, CHUNK_THREADS>;
    __shared__ typename BR::TempStorage tmp;
    uint4 v = flags[(long long)blockIdx.x * CHUNK_THREADS + threadIdx.x];
    int c = BR(tmp).Sum(nz_bytes(v));
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(CHUNK_THREADS)
k_chunk_emit(const uint4 *__restrict__ flags, const int *__restrict__ offs,
             long long *__restrict__ ids) {
    using BS = cub::BlockScan<int, CHUNK_THREADS>;
    __shared__ typename BS::TempStorage tmp;
    long long t = (long long)blockIdx.x * CHUNK_THREADS + threadIdx.x;
    uint4 v = flags[t];
    int ex;
    BS(tmp).ExclusiveSum(nz_bytes(v), ex);
    long long pos = offs[blockIdx.x] + ex;
    unsigned w[4] = {v.x, v.y, v.z, v.w};
    long long base = t * 16;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (((w[q] >> (8 * b)) & 0xffu) != 0u) ids[pos++] = base + 4 * q + b;
}

// --------------------------------------------------- listed-edge records --
__global__ void k_cross_fill(const double *__restrict__ atoms, long long na, GridGeo g,
                             CellList cl, const int *__restrict__ cstart,
                             const int *__restrict__ clist, const uint8_t *__restrict__ inside,
                             const long long *__restrict__ ids, long long ncross,
                             double *__restrict__ alpha_out, double *__restrict__ rp,
                             int8_t *__restrict__ sign, BuildInfo *info) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= ncross) return;
    EdgeRef r = edge_ref(g, ids[s]);
    double xa[3] = {node_coord(g, 0, r.ijk[0]), node_coord(g, 1, r.ijk[1]),
                    node_coord(g, 2, r.ijk[2])};
    double al;
    if (!edge_alpha<false>(atoms, na, cl, cstart, clist, xa, r.d, g.h, al)) {
        atomicOr(&info->err, ERRF_TOO_MANY_BALLS);
        al = 0.0;
    }
    alpha_out[s] = al;
    int ina = inside[r.a], inb = inside[r.b];
    double p[3] = {xa[0], xa[1], xa[2]};
    int sg = 0;
    if (ina && !inb) {
        p[r.d] = xa[r.d] + al * g.h;
        sg = 1;
    } else if (!ina && inb) {
        double xb = node_coord(g, r.d, r.ijk[r.d] + 1);
        p[r.d] = xb - al * g.h;
        sg = -1;
    } else {
        p[r.d] = xa[r.d] + 0.5 * g.h;
    }
    rp[3 * s] = p[0];
    rp[3 * s + 1] = p[1];
    rp[3 * s + 2] = p[2];
    sign[s] = (int8_t)sg;
    if (sg != 0) atomicAdd(&info->nflux, 1ull);
}

// rowstart[r] = first listed edge with id >= r*nx, r = (d*nz + k)*ny + j
__global__ void k_rowstart(const long long *__restrict__ ids, long long ncross, int nx,
                           long long nrows, int *__restrict__ rowstart) {
    long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r > nrows) return;
    long long key = r * nx;
    long long lo = 0, hi = ncross;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (ids[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    rowstart[r] = (int)lo;
}

__global__ void k_count_inside(const uint8_t *__restrict__ inside, long long N, BuildInfo *info) {
    using BR = cub::BlockReduce<unsigned long long, 256>;
    __shared__ typename BR::TempStorage tmp;
    unsigned long long c = 0;
    for (long long a = blockIdx.x * 256ll + threadIdx.x; a < N; a += (long long)gridDim.x * 256)
        c += inside[a];
    c = BR(tmp).Sum(c);
    if (threadIdx.x == 0 && c) atomicAdd(&info->ninside, c);
}

}  // namespace

pb_status upload_atoms(pb_grid *g, const double *atoms, int loc, cudaStream_t s) {
    const long long na = g->na;
    size_t bytes = sizeof(double) * 5 * (size_t)na;
    g->atoms = (double *)dalloc(bytes, s);
    double *aos = (double *)dalloc(bytes, s);
    if (!g->atoms || !aos) {
        dfree(aos, s);
        return PB_ERR_OOM;
    }
    PB_CUDA_TRY(cudaMemcpyAsync(aos, atoms, bytes,
                                loc == PB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    k_aos_to_soa<<<cdiv(na, 256), 256, 0, s>>>(aos, g->atoms, na);
    PB_LAUNCH_CHECK();
    dfree(aos, s);
    return PB_OK;
}

pb_status grid_build(pb_grid *g, const pb_grid_spec *spec, cudaStream_t s) {
    const long long na = g->na;
    // ---- placement + validation (one sync to read the geometry back)
    int auto_place = spec->h == 0.0;
    int nmax = spec->n[0];
    PB_CUDA_TRY(cudaMemsetAsync(g->d_info, 0, sizeof(BuildInfo), s));
    k_prep<<<1, PREP_THREADS, 0, s>>>(g->atoms, na, auto_place, nmax, spec->fill, spec->n[0],
                                      spec->n[1], spec->n[2], spec->origin[0], spec->origin[1],
                                      spec->origin[2], spec->h, g->d_info);
    PB_LAUNCH_CHECK();
    BuildInfo hinfo;
    PB_CUDA_TRY(cudaMemcpyAsync(&hinfo, g->d_info, sizeof(BuildInfo), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo.err & ERRF_ATOM_VALUE) {
        set_error("atoms: non-finite value or non-positive radius");
        return PB_ERR_ARG;
    }
    if (hinfo.err & ERRF_CHARGE_CELL) {
        set_error("a charge's trilinear cell touches the box boundary (grid too small)");
        return PB_ERR_ARG;
    }
    if (!(hinfo.h > 0.0) || !isfinite(hinfo.h)) {
        set_error("grid spacing is not positive");
        return PB_ERR_ARG;
    }
    GridGeo &geo = g->geo;
    geo.nx = spec->n[0];
    geo.ny = spec->n[1];
    geo.nz = spec->n[2];
    geo.N = (long long)geo.nx * geo.ny * geo.nz;
    for (int d = 0; d < 3; ++d) geo.o[d] = hinfo.origin[d];
    geo.h = hinfo.h;
    for (int d = 0; d < 3; ++d)
        g->center[d] = geo.o[d] + 0.5 * (double)((d == 0 ? geo.nx : d == 1 ? geo.ny : geo.nz) - 1) * geo.h;
    const long long N = geo.N;

    // ---- classification
    g->inside = (uint8_t *)dalloc(N, s);
    if (!g->inside) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(g->inside, 0, N, s));
    const unsigned atom_blocks = (unsigned)(na < 65535 ? na : 65535);
    {
        k_classify<<<atom_blocks, 256, 0, s>>>(g->atoms, na, geo, g->inside);
        PB_LAUNCH_CHECK();
    }
    k_count_inside<<<num_sms() * 4, 256, 0, s>>>(g->inside, N, g->d_info);
    PB_LAUNCH_CHECK();

    // ---- atom cell list (cells of side >= rmax + 1.01 h over the balls' box)
    CellList &cl = g->cells;
    cl.cs = hinfo.rmax + 1.01 * geo.h;
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        cl.lo[d] = hinfo.lo[d] - cl.cs;
        cl.dim[d] = (int)((hinfo.hi[d] - cl.lo[d]) / cl.cs) + 2;
        ncell *= cl.dim[d];
    }
    if (ncell > (1ll << 27)) {
        set_error("atom cell list too large (%lld cells)", ncell);
        return PB_ERR_ARG;
    }
    cl.ncell = (int)ncell;
    cl.start = (int *)dalloc(sizeof(int) * (ncell + 1), s);
    cl.atom = (int *)dalloc(sizeof(int) * (na + 1), s);
    int *count = (int *)dalloc(sizeof(int) * (ncell + 1), s);
    int *acell = (int *)dalloc(sizeof(int) * (na + 1), s);
    if (!cl.start || !cl.atom || !count || !acell) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (ncell + 1), s));
    k_cell_count<<<cdiv(na, 256), 256, 0, s>>>(g->atoms, na, cl, acell, count, g->d_info);
    PB_LAUNCH_CHECK();
    k_scan_int<1024><<<1, 1024, 0, s>>>(count, cl.start, (int)ncell);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (ncell + 1), s));
    k_cell_fill<<<cdiv(na, 256), 256, 0, s>>>(acell, na, cl.start, count, cl.atom);
    PB_LAUNCH_CHECK();
    k_cell_sort<<<cdiv(ncell, 128), 128, 0, s>>>(cl.start, cl.atom, (int)ncell);
    PB_LAUNCH_CHECK();
    dfree(count, s);
    dfree(acell, s);

    // ---- listed edges: flags -> ordered compaction -> records
    long long nedge = 3 * N;
    long long nchunks = (nedge + CHUNK_BYTES - 1) / CHUNK_BYTES;
    long long nflags = nchunks * CHUNK_BYTES;
    uint8_t *flags = (uint8_t *)dalloc(nflags, s);
    uint8_t *cov = (uint8_t *)dalloc(nflags, s);
    int *ccount = (int *)dalloc(sizeof(int) * (nchunks + 1), s);
    int *coffs = (int *)dalloc(sizeof(int) * (nchunks + 1), s);
    if (!flags || !cov || !ccount || !coffs) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(flags, 0, nflags, s));
    PB_CUDA_TRY(cudaMemsetAsync(cov, 0, nflags, s));
    if (na > 0) {
        k_edge_cand<<<atom_blocks, 128, 0, s>>>(g->atoms, na, geo, flags, cov);
        PB_LAUNCH_CHECK();
    }
    k_edge_flags<<<(unsigned)nchunks, CHUNK_THREADS, 0, s>>>(g->atoms, na, geo, cl, cl.start,
                                                              cl.atom, g->inside, flags, cov,
                                                              g->d_info);
    PB_LAUNCH_CHECK();
    dfree(cov, s);
    k_chunk_count<<<(unsigned)nchunks, CHUNK_THREADS, 0, s>>>((const uint4 *)flags, ccount);
    PB_LAUNCH_CHECK();
    k_scan_int<1024><<<1, 1024, 0, s>>>(ccount, coffs, (int)nchunks);
    PB_LAUNCH_CHECK();
    int total = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&total, coffs + nchunks, sizeof(int), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaMemcpyAsync(&hinfo, g->d_info, sizeof(BuildInfo), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo.err & ERRF_CELL_OVERFLOW) {
        set_error("internal: atom outside its cell list");
        return PB_ERR_CUDA;
    }
    g->ncross = total;
    long long nc = total > 0 ? total : 1;
    g->cid = (long long *)dalloc(sizeof(long long) * nc, s);
    g->calpha = (double *)dalloc(sizeof(double) * nc, s);
    g->crp = (double *)dalloc(sizeof(double) * 3 * nc, s);
    g->csign = (int8_t *)dalloc(nc, s);
    long long nrows = 3ll * geo.ny * geo.nz;
    g->rowstart = (int *)dalloc(sizeof(int) * (nrows + 1), s);
    if (!g->cid || !g->calpha || !g->crp || !g->csign || !g->rowstart) return PB_ERR_OOM;
    if (total > 0) {
        k_chunk_emit<<<(unsigned)nchunks, CHUNK_THREADS, 0, s>>>((const uint4 *)flags, coffs,
                                                                 g->cid);
        PB_LAUNCH_CHECK();
        k_cross_fill<<<cdiv(total, 256), 256, 0, s>>>(g->atoms, na, geo, cl, cl.start, cl.atom,
                                                      g->inside, g->cid, total, g->calpha,
                                                      g->crp, g->csign, g->d_info);
        PB_LAUNCH_CHECK();
    }
    k_rowstart<<<cdiv(nrows + 1, 256), 256, 0, s>>>(g->cid, total, geo.nx, nrows, g->rowstart);
    PB_LAUNCH_CHECK();
    dfree(flags, s);
    dfree(ccount, s);
    dfree(coffs, s);
    PB_CUDA_TRY(cudaMemcpyAsync(&hinfo, g->d_info, sizeof(BuildInfo), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hinfo.err & ERRF_TOO_MANY_BALLS) {
        set_error("more than %d atom balls meet one listed grid edge", MAX_EDGE_BALLS);
        return PB_ERR_ARG;
    }
    g->nflux = (long long)hinfo.nflux;
    g->ninside = (long long)hinfo.ninside;
    // the surface re-triangulated through the crossing points (first
    // integral of Eq. energy_ion, Sec. 3.3.2): vertex weights and normals
    return mc_surface(g, s);
}

}  // namespace pbg
