// Analytic N-body sums of the energy partition (Sec. 3.3) and of the
// Coulomb / Debye-Hueckel boundary condition (Sec. 2.3).
//
//   Phi_t = sum_i q_i exp(-k r_ti) / r_ti          (k = 0: Coulomb)
//   Psi_t = sum_i q_i (r_t - r_i).n_t / r_ti^3      (dipole kernel, n_t = +-e_d)
//
// FP32 tiled kernel: sources staged in shared memory 256 at a time; each
// position is stored as an FP32 pair (hi + lo) relative to the grid centre so
// the difference r_t - r_i keeps ~46 bits; 1/r from rsqrtf; each tile's
// contributions are summed with Kahan compensation in FP32 and the tile sum
// is added to an FP64 accumulator.
#include <cub/block/block_reduce.cuh>

#include "pb_internal.h"

namespace pbg {

namespace {

constexpr int NB_THREADS = 256;
constexpr int NB_TPT = 2;  // targets per thread

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
enum { TK_BOUNDARY = 0, TK_SURFACE = 1, TK_ATOMS = 2 };

struct TargetDesc {
    int kind;
    GridGeo g;
    double shift[3];
    // surface
    const double *rp;
    const long long *ids;
    const int8_t *sign;
    // atoms
    const double *atoms;
    long long na;
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
    bool active;    // contributes (flux edge / valid index)
};

__device__ __forceinline__ TgtLoad load_target(const TargetDesc &T, long long t) {
    TgtLoad r;
    double p[3] = {0.0, 0.0, 0.0};
    r.active = t < T.count;
    r.n[0] = r.n[1] = r.n[2] = 0.f;
    if (r.active) {
        if (T.kind == TK_BOUNDARY) {
            long long i, j, k;
            boundary_node(T.g, t, i, j, k);
            p[0] = T.g.o[0] + (double)i * T.g.h;
            p[1] = T.g.o[1] + (double)j * T.g.h;
            p[2] = T.g.o[2] + (double)k * T.g.h;
        } else if (T.kind == TK_SURFACE) {
            int sg = T.sign[t];
            if (sg == 0) r.active = false;
            int d = (int)(T.ids[t] / T.g.N);
            r.n[d] = (float)sg;
            p[0] = T.rp[3 * t];
            p[1] = T.rp[3 * t + 1];
            p[2] = T.rp[3 * t + 2];
        } else {
            p[0] = T.atoms[t];
            p[1] = T.atoms[T.na + t];
            p[2] = T.atoms[2 * T.na + t];
        }
    }
    for (int d = 0; d < 3; ++d) {
        double c = p[d] - T.shift[d];
        r.h[d] = (float)c;
        r.l[d] = (float)(c - (double)r.h[d]);
    }
    return r;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// out_phi[t] = scale * sum_i q_i exp(-k r)/r; out_psi[t] = sum_i q_i (r.n)/r^3
// (PSI only for surface targets).  Self pairs (r == 0) are skipped.
template <bool PSI, bool SCREEN>
__global__ void __launch_bounds__(NB_THREADS)
k_nbody(TargetDesc T, const float4 *__restrict__ shi, const float4 *__restrict__ slo,
        long long ns, float kscr, double scale, double *__restrict__ out_phi,
        double *__restrict__ out_psi) {
    __shared__ float4 sh[NB_THREADS], sl[NB_THREADS];
    long long t0 = ((long long)blockIdx.x * NB_THREADS * NB_TPT) + threadIdx.x;
    TgtLoad tg[NB_TPT];
    double acc_phi[NB_TPT], acc_psi[NB_TPT];
#pragma unroll
    for (int u = 0; u < NB_TPT; ++u) {
        tg[u] = load_target(T, t0 + (long long)u * NB_THREADS);
        acc_phi[u] = 0.0;
        acc_psi[u] = 0.0;
    }
    for (long long base = 0; base < ns; base += NB_THREADS) {
        long long si = base + threadIdx.x;
        __syncthreads();
        if (si < ns) {
            sh[threadIdx.x] = shi[si];
            sl[threadIdx.x] = slo[si];
        } else {
            sh[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            sl[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        int m = (int)min((long long)NB_THREADS, ns - base);
        float sp[NB_TPT], cp[NB_TPT], sq[NB_TPT], cq[NB_TPT];
#pragma unroll
        for (int u = 0; u < NB_TPT; ++u) sp[u] = cp[u] = sq[u] = cq[u] = 0.f;
#pragma unroll 4
        for (int q = 0; q < m; ++q) {
            float4 a = sh[q], b = sl[q];
#pragma unroll
            for (int u = 0; u < NB_TPT; ++u) {
                float dx = (tg[u].h[0] - a.x) + (tg[u].l[0] - b.x);
                float dy = (tg[u].h[1] - a.y) + (tg[u].l[1] - b.y);
                float dz = (tg[u].h[2] - a.z) + (tg[u].l[2] - b.z);
                float r2 = dx * dx + dy * dy + dz * dz;
                float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
                float v = a.w * ri;
                if (SCREEN) v *= expf(-kscr * (r2 * ri));
                kahan_add(sp[u], cp[u], v);
                if (PSI) {
                    float dn = dx * tg[u].n[0] + dy * tg[u].n[1] + dz * tg[u].n[2];
                    kahan_add(sq[u], cq[u], v * dn * (ri * ri));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < NB_TPT; ++u) {
            acc_phi[u] += (double)sp[u] - (double)cp[u];
            if (PSI) acc_psi[u] += (double)sq[u] - (double)cq[u];
        }
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

// sum_i q_i Phi_i in a fixed order (one block) -> eacc->ecoul_sum
__global__ void __launch_bounds__(1024)
k_reduce_qphi(const double *__restrict__ atoms, long long na, const double *__restrict__ phi,
              EnergyAcc *eacc) {
    using BR = cub::BlockReduce<double, 1024>;
    __shared__ typename BR::TempStorage tmp;
    double s = 0.0;
    for (long long i = threadIdx.x; i < na; i += 1024) s += atoms[4 * na + i] * phi[i];
    double tot = BR(tmp).Sum(s);
    if (threadIdx.x == 0) eacc->ecoul_sum = tot;
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
    T.atoms = g->atoms;
    T.na = g->na;
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
    k_nbody<true, false><<<cdiv(T.count, NB_THREADS * NB_TPT), NB_THREADS, 0, s>>>(
        T, hi, lo, g->na, 0.f, 1.0, sys->Phi, sys->Psi);
    PB_LAUNCH_CHECK();
    dfree(hi, s);
    dfree(lo, s);
    return PB_OK;
}

pb_status nbody_pairs(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    long long na = g->na > 0 ? g->na : 1;
    if (!sys->ecoul_phi) sys->ecoul_phi = (double *)dalloc(sizeof(double) * na, s);
    if (!sys->ecoul_phi) return PB_ERR_OOM;
    if (g->na == 0) {
        PB_CUDA_TRY(cudaMemsetAsync(&sys->eacc->ecoul_sum, 0, sizeof(double), s));
        return PB_OK;
    }
    float4 *hi, *lo;
    pb_status st = split_sources(sys, s, &hi, &lo);
    if (st != PB_OK) return st;
    TargetDesc T = make_desc(sys, TK_ATOMS);
    T.count = g->na;
    k_nbody<false, false><<<cdiv(T.count, NB_THREADS * NB_TPT), NB_THREADS, 0, s>>>(
        T, hi, lo, g->na, 0.f, 1.0, sys->ecoul_phi, nullptr);
    PB_LAUNCH_CHECK();
    k_reduce_qphi<<<1, 1024, 0, s>>>(g->atoms, g->na, sys->ecoul_phi, sys->eacc);
    PB_LAUNCH_CHECK();
    dfree(hi, s);
    dfree(lo, s);
    return PB_OK;
}

}  // namespace pbg
