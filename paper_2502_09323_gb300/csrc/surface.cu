// Re-triangulated molecular surface for the first integral of Eq.
// energy_ion (Sec. 3.3.2): the surface is rebuilt cell by cell by marching
// cubes whose vertices are the analytic intersection points r_p of the
// crossing edges (end nodes in different media), with the analytic normal of
// the ball surface at each vertex; the integral then takes the vertex rule
// T_j/3 on every triangle, with phi at the vertices from Eq. phi0 (in the
// energy kernel).
//
// One cell's triangles, without a case table: on each face the crossing
// edges are joined in pairs (two crossings: one segment; four, the ambiguous
// face: two segments that each cut off one inside corner, so both cells of a
// face agree and the surface is closed).  Every crossing edge of the cell
// lies on two faces, so the segments close into loops; a loop starts at its
// lowest cell-edge index, first goes to the smaller of that vertex's two
// neighbours, and is cut into the fan (v0, v_m, v_m+1).
//
// k_mc_weight gives every crossing point W = sum of T_j/3 over the triangles
// of its (up to four) cells that have it as a vertex, visiting the cells in
// node order and their triangles in fan order, so each sum is formed in one
// fixed order without atomics.  k_mc_normal finds, through the atom cell
// list, the ball whose sphere passes closest to the point (smallest
// | |r_p - c| - R |, ties to the lower atom index) and takes the unit vector
// from its centre; an FP32 pass first bounds that minimum, so that the FP64
// comparison only visits the candidates that can reach it.  This file is compiled without FMA contraction, so every
// value is reproducible to the bit.
#include <math.h>

#include "pb_internal.h"

namespace pbg {

namespace {

// cell corners: bit 0 = +x, bit 1 = +y, bit 2 = +z.  Cell edges: 0-3 along
// x, 4-7 along y, 8-11 along z (corner pairs below).
__constant__ int8_t c_edge_corner[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                            {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// faces: corners in cyclic order, and the cell edge between corner q and q+1
__constant__ int8_t c_face[6][4] = {{0, 2, 6, 4}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                    {2, 3, 7, 6}, {0, 1, 3, 2}, {4, 5, 7, 6}};
__constant__ int8_t c_face_edge[6][4] = {{4, 10, 6, 8}, {5, 11, 7, 9}, {0, 9, 2, 8},
                                         {1, 11, 3, 10}, {0, 5, 1, 4}, {2, 7, 3, 6}};

// index of edge id in the sorted crossing list (-1 if absent): a binary
// search inside the id's edge row, [rowstart[r], rowstart[r + 1]) with
// r = id / nx
__device__ long long find_edge(const long long *__restrict__ ids, const int *__restrict__ rowstart,
                               int nx, long long id) {
    const long long r = id / nx;
    long long lo = rowstart[r], hi = (long long)rowstart[r + 1] - 1;
    while (lo <= hi) {
        const long long mid = lo + (hi - lo) / 2;
        const long long v = ids[mid];
        if (v == id) return mid;
        if (v < id) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Adds to w, in fan order, T/3 of every triangle of cell (ci, cj, ck) that
// has the cell edge es (the crossing point s) as a vertex.  The cell's
// state lives in registers: the neighbours of each crossed cell edge as
// 4-bit fields (filled in face order, first neighbour first), a loop as a
// string of 4-bit edge indices.
__device__ void mc_cell_acc(const GridGeo &g, const uint8_t *__restrict__ inside,
                            const long long *__restrict__ ids, const int *__restrict__ rowstart,
                            const double *__restrict__ rp, long long ci, long long cj,
                            long long ck, int es, double &w) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const long long n0 = (ck * g.ny + cj) * g.nx + ci;
    auto node = [&](int c) -> long long {
        return n0 + (c & 1) + ((c >> 1) & 1) * sy + ((c >> 2) & 1) * sz;
    };
    int ins = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (inside[node(c)]) ins |= 1 << c;
    if (ins == 0 || ins == 0xff) return;
    unsigned cm = 0;  // crossed cell edges
#pragma unroll
    for (int e = 0; e < 12; ++e)
        if (((ins >> c_edge_corner[e][0]) ^ (ins >> c_edge_corner[e][1])) & 1) cm |= 1u << e;
    if (!((cm >> es) & 1)) return;
    unsigned long long nb0 = 0, nb1 = 0;
    unsigned has0 = 0;
    auto link = [&](int a, int b) {
        if (!((has0 >> a) & 1)) {
            nb0 |= (unsigned long long)b << (4 * a);
            has0 |= 1u << a;
        } else {
            nb1 |= (unsigned long long)b << (4 * a);
        }
    };
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        int crp = 0, m = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (((ins >> c_face[f][q]) ^ (ins >> c_face[f][(q + 1) & 3])) & 1) {
                crp |= q << (2 * m);
                ++m;
            }
        if (m == 2) {
            const int a = c_face_edge[f][crp & 3], b = c_face_edge[f][(crp >> 2) & 3];
            link(a, b);
            link(b, a);
        } else if (m == 4) {
            // cut off each inside corner (corner q lies between face edges q-1 and q)
            const int q0 = ((ins >> c_face[f][0]) & 1) ? 0 : 1;
            const int pa0 = c_face_edge[f][(q0 + 3) & 3], pb0 = c_face_edge[f][q0];
            const int pa1 = c_face_edge[f][(q0 + 1) & 3], pb1 = c_face_edge[f][(q0 + 2) & 3];
            link(pa0, pb0);
            link(pb0, pa0);
            link(pa1, pb1);
            link(pb1, pa1);
        }
    }
    auto vert = [&](int e) -> long long {
        return find_edge(ids, rowstart, g.nx, (long long)(e / 4) * g.N + node(c_edge_corner[e][0]));
    };
    unsigned seen = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
        if (!((cm >> e0) & 1) || ((seen >> e0) & 1)) continue;
        unsigned long long lp = (unsigned long long)e0;
        int len = 1, prev = e0;
        const int f0 = (int)((nb0 >> (4 * e0)) & 15), f1 = (int)((nb1 >> (4 * e0)) & 15);
        int cur = f0 < f1 ? f0 : f1;
        seen |= 1u << e0;
        while (cur != e0 && len < 12) {
            lp |= (unsigned long long)cur << (4 * len);
            ++len;
            seen |= 1u << cur;
            const int a0 = (int)((nb0 >> (4 * cur)) & 15), a1 = (int)((nb1 >> (4 * cur)) & 15);
            const int nx = a0 == prev ? a1 : a0;
            prev = cur;
            cur = nx;
        }
        for (int m = 1; m + 1 < len; ++m) {
            const int ea = (int)(lp & 15), eb = (int)((lp >> (4 * m)) & 15),
                      ec = (int)((lp >> (4 * (m + 1))) & 15);
            if (ea != es && eb != es && ec != es) continue;
            const long long a = vert(ea), b = vert(eb), c = vert(ec);
            if (a < 0 || b < 0 || c < 0) continue;
            const double *p0 = rp + 3 * a, *p1 = rp + 3 * b, *p2 = rp + 3 * c;
            const double u0 = p1[0] - p0[0], u1 = p1[1] - p0[1], u2 = p1[2] - p0[2];
            const double v0 = p2[0] - p0[0], v1 = p2[1] - p0[1], v2 = p2[2] - p0[2];
            const double x = u1 * v2 - u2 * v1;
            const double y = u2 * v0 - u0 * v2;
            const double z = u0 * v1 - u1 * v0;
            w += 0.5 * sqrt((x * x + y * y) + z * z) / 3.0;
        }
    }
}

__global__ void __launch_bounds__(128)
k_mc_weight(GridGeo g, const uint8_t *__restrict__ inside, const long long *__restrict__ ids,
            const int *__restrict__ rowstart, const int8_t *__restrict__ sign,
            const double *__restrict__ rp, long long ncross, double *__restrict__ W) {
    const long long s = blockIdx.x * 128ll + threadIdx.x;
    if (s >= ncross) return;
    double w = 0.0;
    if (sign[s] != 0) {
        const long long id = ids[s];
        const int d = (int)(id / g.N);
        const long long a = id - (long long)d * g.N;
        const long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
        // the (up to) four cells around the edge, in node order; the edge's
        // index in each: x edges 0-3 by (dy + 2 dz), y edges 4-7 by
        // (dx + 2 dz), z edges 8-11 by (dx + 2 dy), offsets from the cell
        for (int v = 0; v < 2; ++v)
            for (int u = 0; u < 2; ++u) {
                long long ci = i, cj = j, ck = k;
                if (d == 0) {
                    cj = j - 1 + u;
                    ck = k - 1 + v;
                } else if (d == 1) {
                    ci = i - 1 + u;
                    ck = k - 1 + v;
                } else {
                    ci = i - 1 + u;
                    cj = j - 1 + v;
                }
                if (ci < 0 || cj < 0 || ck < 0 || ci > g.nx - 2 || cj > g.ny - 2 || ck > g.nz - 2)
                    continue;
                const int ox = (int)(i - ci), oy = (int)(j - cj), oz = (int)(k - ck);
                const int es = d == 0 ? oy + 2 * oz : (d == 1 ? 4 + ox + 2 * oz : 8 + ox + 2 * oy);
                mc_cell_acc(g, inside, ids, rowstart, rp, ci, cj, ck, es, w);
            }
    }
    W[s] = w;
}

// FP32 copies of the atoms relative to the cell list's corner: (x, y, z, R)
__global__ void k_atoms32(const double *__restrict__ atoms, long long na, CellList cl,
                          float4 *__restrict__ a32) {
    const long long i = blockIdx.x * 128ll + threadIdx.x;
    if (i >= na) return;
    a32[i] = make_float4((float)(atoms[i] - cl.lo[0]), (float)(atoms[na + i] - cl.lo[1]),
                         (float)(atoms[2 * na + i] - cl.lo[2]), (float)atoms[3 * na + i]);
}

// |r - c| - R in FP32 differs from the FP64 value by at most about
// 4 * 2^-24 * X, X the largest coordinate relative to the cell list's corner
// (each rounding of a coordinate to FP32 costs 2^-24 X, the difference and
// the distance add rounding of their own); a candidate whose FP32 value
// exceeds the FP32 minimum by more than twice that bound can be neither the
// FP64 minimum nor tied with it.  The margin passed in is several times that.

__global__ void __launch_bounds__(128)
k_mc_normal(const double *__restrict__ atoms, const float4 *__restrict__ a32, long long na,
            CellList cl, float margin, const int8_t *__restrict__ sign,
            const double *__restrict__ rp, long long ncross, double *__restrict__ nrm) {
    const long long s = blockIdx.x * 128ll + threadIdx.x;
    if (s >= ncross) return;
    double o0 = 0.0, o1 = 0.0, o2 = 0.0;
    if (sign[s] != 0) {
        const double p0 = rp[3 * s], p1 = rp[3 * s + 1], p2 = rp[3 * s + 2];
        const double p[3] = {p0, p1, p2};
        int cc[3];
        for (int q = 0; q < 3; ++q) {
            const double u = floor((p[q] - cl.lo[q]) / cl.cs);
            cc[q] = (u < -4.0) ? -4 : ((u > (double)cl.dim[q] + 4.0) ? cl.dim[q] + 4 : (int)u);
        }
        const float f0 = (float)(p0 - cl.lo[0]), f1 = (float)(p1 - cl.lo[1]),
                    f2 = (float)(p2 - cl.lo[2]);
        // pass 1: the smallest FP32 deviation
        float m32 = INFINITY;
        for (int cz = cc[2] - 1; cz <= cc[2] + 1; ++cz) {
            if (cz < 0 || cz >= cl.dim[2]) continue;
            for (int cy = cc[1] - 1; cy <= cc[1] + 1; ++cy) {
                if (cy < 0 || cy >= cl.dim[1]) continue;
                for (int cx = cc[0] - 1; cx <= cc[0] + 1; ++cx) {
                    if (cx < 0 || cx >= cl.dim[0]) continue;
                    const int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
                    for (int q = cl.start[cid]; q < cl.start[cid + 1]; ++q) {
                        const float4 a = a32[cl.atom[q]];
                        const float dx = f0 - a.x, dy = f1 - a.y, dz = f2 - a.z;
                        m32 = fminf(m32, fabsf(sqrtf(dx * dx + dy * dy + dz * dz) - a.w));
                    }
                }
            }
        }
        // pass 2: the FP64 comparison, in the same order, over the
        // candidates that can win
        const float lim = m32 + margin;
        long long best = -1;
        double bdev = 0.0, bd = 0.0;
        for (int cz = cc[2] - 1; cz <= cc[2] + 1; ++cz) {
            if (cz < 0 || cz >= cl.dim[2]) continue;
            for (int cy = cc[1] - 1; cy <= cc[1] + 1; ++cy) {
                if (cy < 0 || cy >= cl.dim[1]) continue;
                for (int cx = cc[0] - 1; cx <= cc[0] + 1; ++cx) {
                    if (cx < 0 || cx >= cl.dim[0]) continue;
                    const int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
                    for (int q = cl.start[cid]; q < cl.start[cid + 1]; ++q) {
                        const long long at = cl.atom[q];
                        const float4 a = a32[at];
                        const float ex = f0 - a.x, ey = f1 - a.y, ez = f2 - a.z;
                        if (fabsf(sqrtf(ex * ex + ey * ey + ez * ez) - a.w) > lim) continue;
                        const double dx = p0 - atoms[at], dy = p1 - atoms[na + at],
                                     dz = p2 - atoms[2 * na + at];
                        const double dd = sqrt((dx * dx + dy * dy) + dz * dz);
                        const double dev = fabs(dd - atoms[3 * na + at]);
                        if (best < 0 || dev < bdev || (dev == bdev && at < best)) {
                            best = at;
                            bdev = dev;
                            bd = dd;
                        }
                    }
                }
            }
        }
        if (best >= 0) {
            o0 = (p0 - atoms[best]) / bd;
            o1 = (p1 - atoms[na + best]) / bd;
            o2 = (p2 - atoms[2 * na + best]) / bd;
        }
    }
    nrm[3 * s] = o0;
    nrm[3 * s + 1] = o1;
    nrm[3 * s + 2] = o2;
}

}  // namespace

// Vertex weights and normals of the re-triangulated surface, from the
// uniform grid pass (the grid itself, or an octree's finest lattice).
pb_status mc_surface(pb_grid *g, cudaStream_t s) {
    const long long nc = g->ncross;
    g->mc_w = (double *)dalloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1), s);
    g->mc_n = (double *)dalloc(sizeof(double) * 3 * (size_t)(nc > 0 ? nc : 1), s);
    if (!g->mc_w || !g->mc_n) return PB_ERR_OOM;
    if (nc == 0) return PB_OK;
    k_mc_weight<<<cdiv(nc, 128), 128, 0, s>>>(g->geo, g->inside, g->cid, g->rowstart, g->csign,
                                              g->crp, nc, g->mc_w);
    PB_LAUNCH_CHECK();
    float4 *a32 = (float4 *)dalloc(sizeof(float4) * (size_t)(g->na > 0 ? g->na : 1), s);
    if (!a32) return PB_ERR_OOM;
    if (g->na > 0) {
        k_atoms32<<<cdiv(g->na, 128), 128, 0, s>>>(g->atoms, g->na, g->cells, a32);
        PB_LAUNCH_CHECK();
    }
    // coordinates of the searched points and atoms stay within the cell
    // list's box widened by four cells on each side
    const CellList &cl = g->cells;
    double ext = 0.0;
    for (int q = 0; q < 3; ++q) ext = fmax(ext, (double)(cl.dim[q] + 8) * cl.cs);
    const float margin = (float)(1e-3 + 64.0 * ext * 5.9604644775390625e-8);
    k_mc_normal<<<cdiv(nc, 128), 128, 0, s>>>(g->atoms, a32, g->na, cl, margin, g->csign, g->crp,
                                              nc, g->mc_n);
    PB_LAUNCH_CHECK();
    dfree(a32, s);
    return PB_OK;
}

}  // namespace pbg
