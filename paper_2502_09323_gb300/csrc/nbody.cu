// Analytic N-body sums of the energy partition (Sec. 3.3) and of the
// Coulomb / Debye-Hueckel boundary condition (Sec. 2.3).
//
//   Phi_t = sum_i q_i exp(-k r_ti) / r_ti          (k = 0: Coulomb)
//   Psi_t = sum_i q_i (r_t - r_i).n_t / r_ti^3      (dipole kernel, n_t = +-e_d,
//                                                    or the analytic surface normal)
//
// FP32 tiled kernel: sources staged in shared memory 256 at a time; each
// position is stored as an FP32 pair (hi + lo) relative to the grid centre so
// the difference r_t - r_i keeps ~46 bits; 1/r from rsqrtf; a tile's
// contributions are summed in groups of 16 in plain FP32, the group sums with
// Kahan compensation in FP32, and the tile sum is added to an FP64
// accumulator.  A thread's two targets share each
// instruction through the packed FP32x2 arithmetic of sm_100-class GPUs.
// It serves the surface terms Phi_p, Psi_p at the crossing points.
//
// FP64 kernels: the boundary values (they enter the linear system) and the
// Coulomb energy sum_{i<j} q_i q_j / r_ij (a net value of large terms of
// either sign), each summed in a fixed order.
#include <cub/block/block_reduce.cuh>

#include "pb_internal.h"

namespace pbg {

namespace {

constexpr int NB_THREADS = 256;
constexpr int NB_TPT = 2;  // targets per thread
constexpr int NB_GRP = 16; // sources per plainly summed group
// largest coordinate offset (A) of a block's targets from its first target
// for the per-block origin form of the differences
constexpr double NB_ORIGIN_EXT = 8.0;

struct SrcHi {
    float x, y, z, q;
};
struct SrcLo {
    float x, y, z, pad;
};

__global__ void k_split_atoms(const double *__restrict__ atoms, long long na, double cx, double cy,
                              double cz, float4 *__restrict__ hi, float4 *__restrict__ lo) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= na) return;
    double c[3] = {atoms[i] - cx, atoms[na + i] - cy, atoms[2 * na + i] - cz};
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
        h[d] = (float)c[d];
        l[d] = (float)(c[d] - (double)h[d]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], (float)atoms[4 * na + i]);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// Target kinds
enum { TK_BOUNDARY = 0, TK_SURFACE = 1 };

struct TargetDesc {
    int kind;
    GridGeo g;
    double shift[3];
    // surface
    const double *rp;
    const long long *ids;
    const int8_t *sign;
    const double *nrm2; // optional second normal per target (PSI2): 3 per target
    long long count;
};

__device__ __forceinline__ void boundary_node(const GridGeo &g, long long b, long long &i,
                                              long long &j, long long &k) {
    long long nxy = (long long)g.nx * g.ny;
    if (b < nxy) {
        i = b % g.nx;
        j = b / g.nx;
        k = 0;
        return;
    }
    if (b < 2 * nxy) {
        b -= nxy;
        i = b % g.nx;
        j = b / g.nx;
        k = g.nz - 1;
        return;
    }
    b -= 2 * nxy;
    long long ring = 2ll * g.nx + 2ll * (g.ny - 2);
    k = 1 + b / ring;
    long long q = b % ring;
    if (q < g.nx) {
        i = q;
        j = 0;
    } else if (q < 2ll * g.nx) {
        i = q - g.nx;
        j = g.ny - 1;
    } else {
        long long q2 = q - 2ll * g.nx;
        if (q2 < g.ny - 2) {
            i = 0;
            j = 1 + q2;
        } else {
            i = g.nx - 1;
            j = 1 + q2 - (g.ny - 2);
        }
    }
}

struct TgtLoad {
    float h[3], l[3];
    float n[3];     // unit normal for Psi (surface targets)
    float n2[3];    // second normal (the analytic surface normal) when given
    bool active;    // contributes (flux edge / valid index)
};

__device__ __forceinline__ TgtLoad load_target(const TargetDesc &T, long long t) {
    TgtLoad r;
    double p[3] = {0.0, 0.0, 0.0};
    r.active = t < T.count;
    r.n[0] = r.n[1] = r.n[2] = 0.f;
    r.n2[0] = r.n2[1] = r.n2[2] = 0.f;
    if (r.active) {
        if (T.kind == TK_BOUNDARY) {
            long long i, j, k;
            boundary_node(T.g, t, i, j, k);
            p[0] = T.g.o[0] + (double)i * T.g.h;
            p[1] = T.g.o[1] + (double)j * T.g.h;
            p[2] = T.g.o[2] + (double)k * T.g.h;
        } else {
            int sg = T.sign[t];
            if (sg == 0) r.active = false;
            int d = (int)(T.ids[t] / T.g.N);
            r.n[d] = (float)sg;
            if (T.nrm2)
                for (int d = 0; d < 3; ++d) r.n2[d] = (float)T.nrm2[3 * t + d];
            p[0] = T.rp[3 * t];
            p[1] = T.rp[3 * t + 1];
            p[2] = T.rp[3 * t + 2];
        }
    }
    for (int d = 0; d < 3; ++d) {
        double c = p[d] - T.shift[d];
        r.h[d] = (float)c;
        r.l[d] = (float)(c - (double)r.h[d]);
    }
    return r;
}

// Packed FP32 pair: lane .x works for the thread's first target, .y for its
// second (one FP32x2 instruction does both).
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 v) {
    float2 y = sub2(v, c);
    float2 t = __fadd2_rn(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
}

// The source tiles of one block: per-pair work, group sums and tile sums as
// described above, accumulated into acc_* (FP64).
// ORIGIN: the block's targets lie within NB_ORIGIN_EXT of its first target
// o, and th holds their positions relative to o as single FP32 values (tl
// unused); each source is staged once per tile as its FP32 position relative
// to o, (hi - o_hi) + (lo - o_lo), so that a difference takes one FP32
// operation instead of three.  Near sources (at least one atom radius away
// from a point of the molecular surface) then keep about 15 u of relative
// accuracy in r, far ones about u.
template <bool PSI, bool SCREEN, bool PSI2, int AXIS, bool ORIGIN>
__device__ __forceinline__ void nb_tiles(float4 (*sp4)[4], const float4 *__restrict__ shi,
                                         const float4 *__restrict__ slo, long long ns, float kscr,
                                         const float (&oh)[3], const float (&ol)[3],
                                         const float2 (&th)[3], const float2 (&tl)[3],
                                         const float2 (&tn)[3], const float2 (&tn2)[3],
                                         double (&acc_phi)[NB_TPT], double (&acc_psi)[NB_TPT],
                                         double (&acc_psi2)[NB_TPT]) {
    for (long long base = 0; base < ns; base += NB_THREADS) {
        long long si = base + threadIdx.x;
        __syncthreads();
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (si < ns) {
            a = shi[si];
            b = slo[si];
        }
        if (ORIGIN) {
            const float rx = (a.x - oh[0]) + (b.x - ol[0]), ry = (a.y - oh[1]) + (b.y - ol[1]),
                        rz = (a.z - oh[2]) + (b.z - ol[2]);
            sp4[threadIdx.x][0] = make_float4(rx, rx, ry, ry);
            sp4[threadIdx.x][1] = make_float4(rz, rz, a.w, a.w);
        } else {
            sp4[threadIdx.x][0] = make_float4(a.x, a.x, a.y, a.y);
            sp4[threadIdx.x][1] = make_float4(a.z, a.z, a.w, a.w);
            sp4[threadIdx.x][2] = make_float4(b.x, b.x, b.y, b.y);
            sp4[threadIdx.x][3] = make_float4(b.z, b.z, 0.f, 0.f);
        }
        __syncthreads();
        int m = (int)min((long long)NB_THREADS, ns - base);
        float2 sp = bc2(0.f), cp = bc2(0.f), sq = bc2(0.f), cq = bc2(0.f), s2 = bc2(0.f),
               c2 = bc2(0.f);
        // groups of NB_GRP sources are summed plainly in FP32 (rounding error
        // below (NB_GRP - 1) u of the group's absolute sum) and each group
        // sum enters the tile sum with Kahan compensation
        for (int q0 = 0; q0 < m; q0 += NB_GRP) {
            const int q1 = min(q0 + NB_GRP, m);
            float2 gp = bc2(0.f), gq = bc2(0.f), g2 = bc2(0.f);
#pragma unroll 4
            for (int q = q0; q < q1; ++q) {
                const float4 p0 = sp4[q][0], p1 = sp4[q][1];
                float2 dx, dy, dz;
                if (ORIGIN) {
                    dx = sub2(th[0], make_float2(p0.x, p0.y));
                    dy = sub2(th[1], make_float2(p0.z, p0.w));
                    dz = sub2(th[2], make_float2(p1.x, p1.y));
                } else {
                    const float4 p2 = sp4[q][2], p3 = sp4[q][3];
                    dx = __fadd2_rn(sub2(th[0], make_float2(p0.x, p0.y)),
                                    sub2(tl[0], make_float2(p2.x, p2.y)));
                    dy = __fadd2_rn(sub2(th[1], make_float2(p0.z, p0.w)),
                                    sub2(tl[1], make_float2(p2.z, p2.w)));
                    dz = __fadd2_rn(sub2(th[2], make_float2(p1.x, p1.y)),
                                    sub2(tl[2], make_float2(p3.x, p3.y)));
                }
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 ri = make_float2(r2.x > 0.f ? rsqrtf(r2.x) : 0.f,
                                              r2.y > 0.f ? rsqrtf(r2.y) : 0.f);
                float2 v = __fmul2_rn(make_float2(p1.z, p1.w), ri);
                if (SCREEN) {
                    v.x *= expf(-kscr * (r2.x * ri.x));
                    v.y *= expf(-kscr * (r2.y * ri.y));
                }
                gp = __fadd2_rn(gp, v);
                if (PSI) {
                    // Psi along n: the general dot product, or, for a
                    // block whose targets all lie on edges along AXIS (n =
                    // +-e_AXIS), that coordinate difference (sign applied to
                    // the total)
                    const float2 dn =
                        AXIS == 0 ? dx
                                  : (AXIS == 1 ? dy
                                               : (AXIS == 2 ? dz
                                                            : __ffma2_rn(dz, tn[2],
                                                                         __ffma2_rn(dy, tn[1],
                                                                                    __fmul2_rn(dx, tn[0])))));
                    const float2 vr2 = __fmul2_rn(v, __fmul2_rn(ri, ri));
                    gq = __ffma2_rn(vr2, dn, gq);
                    if (PSI2) {
                        const float2 dn2 = __ffma2_rn(
                            dz, tn2[2], __ffma2_rn(dy, tn2[1], __fmul2_rn(dx, tn2[0])));
                        g2 = __ffma2_rn(vr2, dn2, g2);
                    }
                }
            }
            kahan_add2(sp, cp, gp);
            if (PSI) kahan_add2(sq, cq, gq);
            if (PSI2) kahan_add2(s2, c2, g2);
        }
        acc_phi[0] += (double)sp.x - (double)cp.x;
        acc_phi[1] += (double)sp.y - (double)cp.y;
        if (PSI) {
            acc_psi[0] += (double)sq.x - (double)cq.x;
            acc_psi[1] += (double)sq.y - (double)cq.y;
        }
        if (PSI2) {
            acc_psi2[0] += (double)s2.x - (double)c2.x;
            acc_psi2[1] += (double)s2.y - (double)c2.y;
        }
    }
}

// out_phi[t] = scale * sum_i q_i exp(-k r)/r; out_psi[t] = sum_i q_i (r.n)/r^3
// (PSI only for surface targets); with PSI2 also out_psi2[t] along the
// target's second normal, from the same pairs.  Self pairs (r == 0) are skipped.  Each
// thread holds two targets in the two halves of FP32x2 registers; the
// sources are staged in shared memory already duplicated into (v, v) pairs.
static_assert(NB_TPT == 2, "two targets per thread, one per FP32x2 half");
template <bool PSI, bool SCREEN, bool PSI2 = false>
__global__ void __launch_bounds__(NB_THREADS)
k_nbody(TargetDesc T, const float4 *__restrict__ shi, const float4 *__restrict__ slo,
        long long ns, float kscr, double scale, double *__restrict__ out_phi,
        double *__restrict__ out_psi, double *__restrict__ out_psi2 = nullptr) {
    // per source: (hx,hx,hy,hy) (hz,hz,q,q) (lx,lx,ly,ly) (lz,lz,0,0)
    __shared__ float4 sp4[NB_THREADS][4];
    long long t0 = ((long long)blockIdx.x * NB_THREADS * NB_TPT) + threadIdx.x;
    TgtLoad tg[NB_TPT];
    double acc_phi[NB_TPT], acc_psi[NB_TPT], acc_psi2[NB_TPT];
#pragma unroll
    for (int u = 0; u < NB_TPT; ++u) {
        tg[u] = load_target(T, t0 + (long long)u * NB_THREADS);
        acc_phi[u] = 0.0;
        acc_psi[u] = 0.0;
        acc_psi2[u] = 0.0;
    }
    float2 th[3], tl[3], tn[3], tn2[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        th[d] = make_float2(tg[0].h[d], tg[1].h[d]);
        tl[d] = make_float2(tg[0].l[d], tg[1].l[d]);
        tn[d] = make_float2(tg[0].n[d], tg[1].n[d]);
        tn2[d] = make_float2(tg[0].n2[d], tg[1].n2[d]);
    }
    // a block whose targets all lie on edges of one direction (the
    // crossing list is ordered by direction) takes the axis form of Psi
    int axis = -1;
    if (PSI && T.kind == TK_SURFACE) {
        const long long tb = (long long)blockIdx.x * NB_THREADS * NB_TPT;
        const int dref = (int)(T.ids[tb] / T.g.N);
        bool same = true;
#pragma unroll
        for (int u = 0; u < NB_TPT; ++u) {
            const long long t = t0 + (long long)u * NB_THREADS;
            if (t < T.count && (int)(T.ids[t] / T.g.N) != dref) same = false;
        }
        if (__syncthreads_and(same)) axis = dref;
    }
    // a block whose surface targets all lie within NB_ORIGIN_EXT of its
    // first target takes the differences from that origin
    bool origin = false;
    float oh[3] = {0.f, 0.f, 0.f}, ol[3] = {0.f, 0.f, 0.f};
    if (T.kind == TK_SURFACE) {
        const long long tb = (long long)blockIdx.x * NB_THREADS * NB_TPT;
        double o[3], rel[NB_TPT][3];
        bool near = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) o[d] = T.rp[3 * tb + d];
#pragma unroll
        for (int u = 0; u < NB_TPT; ++u) {
            const long long t = t0 + (long long)u * NB_THREADS;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                rel[u][d] = t < T.count ? T.rp[3 * t + d] - o[d] : 0.0;
                if (!(fabs(rel[u][d]) <= NB_ORIGIN_EXT)) near = false;
            }
        }
        if (__syncthreads_and(near)) {
            origin = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double oc = o[d] - T.shift[d];  // the sources are relative to the shift
                oh[d] = (float)oc;
                ol[d] = (float)(oc - (double)oh[d]);
                th[d] = make_float2((float)rel[0][d], (float)rel[1][d]);
            }
        }
    }
#define PB_NB_TILES(AX)                                                                          \
    (origin ? nb_tiles<PSI, SCREEN, PSI2, AX, true>(sp4, shi, slo, ns, kscr, oh, ol, th, tl, tn, \
                                                     tn2, acc_phi, acc_psi, acc_psi2)            \
            : nb_tiles<PSI, SCREEN, PSI2, AX, false>(sp4, shi, slo, ns, kscr, oh, ol, th, tl, tn, \
                                                      tn2, acc_phi, acc_psi, acc_psi2))
    switch (axis) {
        case 0: PB_NB_TILES(0); break;
        case 1: PB_NB_TILES(1); break;
        case 2: PB_NB_TILES(2); break;
        default: PB_NB_TILES(-1);
    }
#undef PB_NB_TILES
    if (PSI && axis >= 0) {
        // n = sign e_axis: the one nonzero component is the sign
#pragma unroll
        for (int u = 0; u < NB_TPT; ++u)
            acc_psi[u] *= (double)(tg[u].n[0] + tg[u].n[1] + tg[u].n[2]);
    }
#pragma unroll
    for (int u = 0; u < NB_TPT; ++u) {
        long long t = t0 + (long long)u * NB_THREADS;
        if (t >= T.count) continue;
        if (T.kind == TK_BOUNDARY) {
            long long i, j, k;
            boundary_node(T.g, t, i, j, k);
            out_phi[(k * T.g.ny + j) * T.g.nx + i] = scale * acc_phi[u];
        } else {
            out_phi[t] = tg[u].active ? scale * acc_phi[u] : 0.0;
            if (PSI) out_psi[t] = tg[u].active ? acc_psi[u] : 0.0;
            if (PSI2) out_psi2[t] = tg[u].active ? acc_psi2[u] : 0.0;
        }
    }
}

// Boundary values in FP64: they enter the linear system itself, so they are
// summed exactly in double precision (atoms staged in shared memory).
__global__ void __launch_bounds__(NB_THREADS)
k_boundary64(GridGeo g, const double *__restrict__ atoms, long long na, long long count, double k,
             double scale, double *__restrict__ bc) {
    __shared__ double sx[NB_THREADS], sy[NB_THREADS], sz[NB_THREADS], sq[NB_THREADS];
    long long t = blockIdx.x * (long long)NB_THREADS + threadIdx.x;
    double p[3] = {0.0, 0.0, 0.0};
    long long i = 0, j = 0, kk = 0;
    if (t < count) {
        boundary_node(g, t, i, j, kk);
        p[0] = g.o[0] + (double)i * g.h;
        p[1] = g.o[1] + (double)j * g.h;
        p[2] = g.o[2] + (double)kk * g.h;
    }
    double acc = 0.0;
    for (long long base = 0; base < na; base += NB_THREADS) {
        long long si = base + threadIdx.x;
        __syncthreads();
        if (si < na) {
            sx[threadIdx.x] = atoms[si];
            sy[threadIdx.x] = atoms[na + si];
            sz[threadIdx.x] = atoms[2 * na + si];
            sq[threadIdx.x] = atoms[4 * na + si];
        }
        __syncthreads();
        int m = (int)min((long long)NB_THREADS, na - base);
        for (int q = 0; q < m; ++q) {
            double dx = p[0] - sx[q], dy = p[1] - sy[q], dz = p[2] - sz[q];
            double r = sqrt((dx * dx + dy * dy) + dz * dz);
            acc += (k > 0.0 ? sq[q] * exp(-k * r) : sq[q]) / r;
        }
    }
    if (t < count) bc[(kk * g.ny + j) * g.nx + i] = scale * acc;
}

// Coulomb pair sum sum_{i<j} q_i q_j / r_ij in FP64 (the energy is a
// difference of large sums of either sign, so its terms are kept exact to
// rounding).  Atoms in tiles of PT; block (a, b) of the nt x nt grid, a <= b,
// takes the pairs i in tile a, j in tile b (j > i when a == b): thread t holds
// atom i, tile b is staged in shared memory and taken in ascending order,
// 1/r from the double-precision rsqrt.  The block's total goes to
// part[b * nt + a] (zero for a > b); one block then adds the partials in
// index order, so the sum is the same on every run.
constexpr int PT = 128;

__global__ void __launch_bounds__(PT)
k_pairs64(const double *__restrict__ atoms, long long na, double *__restrict__ part) {
    __shared__ double sx[PT], sy[PT], sz[PT], sq[PT];
    using BR = cub::BlockReduce<double, PT>;
    __shared__ typename BR::TempStorage tmp;
    const int a = blockIdx.x, b = blockIdx.y, nt = gridDim.x;
    if (a > b) {
        if (threadIdx.x == 0) part[(long long)b * nt + a] = 0.0;
        return;
    }
    const long long i = (long long)a * PT + threadIdx.x;
    const long long j0 = (long long)b * PT, js = j0 + threadIdx.x;
    if (js < na) {
        sx[threadIdx.x] = atoms[js];
        sy[threadIdx.x] = atoms[na + js];
        sz[threadIdx.x] = atoms[2 * na + js];
        sq[threadIdx.x] = atoms[4 * na + js];
    }
    __syncthreads();
    double mine = 0.0;
    if (i < na) {
        const double px = atoms[i], py = atoms[na + i], pz = atoms[2 * na + i];
        const int m = (int)min((long long)PT, na - j0);
        const int q0 = a == b ? threadIdx.x + 1 : 0;  // j > i on the diagonal tile
        double acc = 0.0;
        for (int q = q0; q < m; ++q) {
            const double dx = px - sx[q], dy = py - sy[q], dz = pz - sz[q];
            const double r2 = (dx * dx + dy * dy) + dz * dz;
            if (r2 > 0.0) acc += sq[q] * rsqrt(r2);
        }
        mine = atoms[4 * na + i] * acc;
    }
    const double tot = BR(tmp).Sum(mine);
    if (threadIdx.x == 0) part[(long long)b * nt + a] = tot;
}

// 2 sum_{i<j} (the sum over i of q_i Phi_i) from the pair partials, in index
// order -> eacc->ecoul_sum
__global__ void __launch_bounds__(1024)
k_reduce_pairs(const double *__restrict__ part, long long n, EnergyAcc *eacc) {
    using BR = cub::BlockReduce<double, 1024>;
    __shared__ typename BR::TempStorage tmp;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += 1024) s += part[i];
    double tot = BR(tmp).Sum(s);
    if (threadIdx.x == 0) eacc->ecoul_sum = 2.0 * tot;
}

pb_status split_sources(pb_system *sys, cudaStream_t s, float4 **hi, float4 **lo) {
    pb_grid *g = sys->g;
    long long na = g->na > 0 ? g->na : 1;
    *hi = (float4 *)dalloc(sizeof(float4) * na, s);
    *lo = (float4 *)dalloc(sizeof(float4) * na, s);
    if (!*hi || !*lo) return PB_ERR_OOM;
    if (g->na > 0) {
        k_split_atoms<<<cdiv(g->na, 256), 256, 0, s>>>(g->atoms, g->na, g->center[0], g->center[1],
                                                       g->center[2], *hi, *lo);
        PB_LAUNCH_CHECK();
    }
    return PB_OK;
}

TargetDesc make_desc(pb_system *sys, int kind) {
    pb_grid *g = sys->g;
    TargetDesc T;
    T.kind = kind;
    T.g = g->geo;
    for (int d = 0; d < 3; ++d) T.shift[d] = g->center[d];
    T.rp = g->crp;
    T.ids = g->cid;
    T.sign = g->csign;
    T.nrm2 = nullptr;
    T.count = 0;
    return T;
}

}  // namespace

pb_status nbody_boundary(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    const GridGeo &geo = g->geo;
    PB_CUDA_TRY(cudaMemsetAsync(sys->bc, 0, sizeof(double) * geo.N, s));
    if (sys->p.bc == PB_BC_ZERO || g->na == 0) return PB_OK;
    long long count =
        2ll * geo.nx * geo.ny + (long long)(geo.nz - 2) * (2ll * geo.nx + 2ll * (geo.ny - 2));
    double scale = sys->lB / sys->p.eps_out;
    double k = sys->p.bc == PB_BC_DH ? sys->kD : 0.0;
    k_boundary64<<<cdiv(count, NB_THREADS), NB_THREADS, 0, s>>>(geo, g->atoms, g->na, count, k,
                                                                scale, sys->bc);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

pb_status nbody_surface(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    long long nc = g->ncross > 0 ? g->ncross : 1;
    if (!sys->Phi) sys->Phi = (double *)dalloc(sizeof(double) * nc, s);
    if (!sys->Psi) sys->Psi = (double *)dalloc(sizeof(double) * nc, s);
    if (!sys->Phi || !sys->Psi) return PB_ERR_OOM;
    if (g->ncross == 0) return PB_OK;
    float4 *hi, *lo;
    pb_status st = split_sources(sys, s, &hi, &lo);
    if (st != PB_OK) return st;
    TargetDesc T = make_desc(sys, TK_SURFACE);
    T.count = g->ncross;
    // Psi along the re-triangulated surface's analytic normals (first
    // integral of Eq. energy_ion, Sec. 3.3.2) comes from the same pairs as
    // Phi and Psi
    if (!sys->PsiN) sys->PsiN = (double *)dalloc(sizeof(double) * nc, s);
    if (!sys->PsiN) return PB_ERR_OOM;
    T.nrm2 = g->mc_n;
    k_nbody<true, false, true><<<cdiv(T.count, NB_THREADS * NB_TPT), NB_THREADS, 0, s>>>(
        T, hi, lo, g->na, 0.f, 1.0, sys->Phi, sys->Psi, sys->PsiN);
    PB_LAUNCH_CHECK();
    dfree(hi, s);
    dfree(lo, s);
    return PB_OK;
}

pb_status nbody_pairs(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    if (g->na <= 1) {
        PB_CUDA_TRY(cudaMemsetAsync(&sys->eacc->ecoul_sum, 0, sizeof(double), s));
        return PB_OK;
    }
    const long long nt = cdiv(g->na, PT);
    if (nt > 8192) {  // the partials grow as nt^2 (512 MB at this limit)
        set_error("too many atoms for the Coulomb pair sum (%lld; at most %d)",
                  (long long)g->na, 8192 * PT);
        return PB_ERR_ARG;
    }
    double *part = (double *)dalloc(sizeof(double) * nt * nt, s);
    if (!part) return PB_ERR_OOM;
    k_pairs64<<<dim3((unsigned)nt, (unsigned)nt), PT, 0, s>>>(g->atoms, g->na, part);
    PB_LAUNCH_CHECK();
    k_reduce_pairs<<<1, 1024, 0, s>>>(part, nt * nt, sys->eacc);
    PB_LAUNCH_CHECK();
    dfree(part, s);
    return PB_OK;
}

}  // namespace pbg
