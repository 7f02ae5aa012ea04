// Coefficient assembly and right-hand side.
//
// Compiled with --fmad=false so the FP64 coefficients and the charge deposit
// are reproducible to the bit (each expression evaluated as written).
//
// Sec. 3.1: with vertex quadrature the Nedelec mass matrix is diagonal and
//   static condensation leaves the 7-point operator A = G^T W G + C, W_e the
//   edge weight eps_e h, C_kk = eps_s k_D^2 h^3 at solvent nodes (the ionic
//   term c = eps_s k_D^2 chi_s of Sec. 2.1 lumped on the node).
// Sec. 3.2 (Eq. WHA): 1/eps_e = alpha/eps_m + (1 - alpha)/eps_s.
// Eq. RVop: f_k = R(w_k) = sum_i q_i w_k(r_i), times 4 pi l_B in reduced units,
//   plus W_e phi_b for every edge that reaches a Dirichlet node.
#include <math.h>

#include "pb_internal.h"

namespace pbg {

namespace {

__device__ __forceinline__ bool is_bnd(const GridGeo &g, long long i, long long j, long long k) {
    return i == 0 || j == 0 || k == 0 || i == g.nx - 1 || j == g.ny - 1 || k == g.nz - 1;
}

// Pure-medium weights for every existing edge; the code byte of the padded
// FP32 layout starts as the solute bit.
__global__ void k_coef_pure(const uint8_t *__restrict__ inside, GridGeo g, PadGeo p,
                            double w_in, double w_out, double *__restrict__ Wx,
                            double *__restrict__ Wy, double *__restrict__ Wz,
                            uint8_t *__restrict__ code) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    int in = inside[a];
    double w = in ? w_in : w_out;
    Wx[a] = (i < g.nx - 1) ? w : 0.0;
    Wy[a] = (j < g.ny - 1) ? w : 0.0;
    Wz[a] = (k < g.nz - 1) ? w : 0.0;
    code[(k * g.ny + j) * p.sx + i] = (uint8_t)in;
}

// Listed edges: WHA weight; FP32 copy for the compressed operator; flag bit
// (1 + d) of the low node's code byte.
__global__ void k_coef_special(const long long *__restrict__ ids, const double *__restrict__ alpha,
                               long long ncross, GridGeo g, PadGeo p, double eps_in,
                               double eps_out, double *__restrict__ Wx, double *__restrict__ Wy,
                               double *__restrict__ Wz, float *__restrict__ wx32,
                               float *__restrict__ wy32, float *__restrict__ wz32,
                               uint8_t *__restrict__ code) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= ncross) return;
    long long e = ids[s];
    int d = (int)(e / g.N);
    long long a = e - (long long)d * g.N;
    double al = alpha[s];
    double w = 1.0 / (al / eps_in + (1.0 - al) / eps_out) * g.h;
    double *W = d == 0 ? Wx : (d == 1 ? Wy : Wz);
    W[a] = w;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    long long pa = (k * g.ny + j) * p.sx + i;
    float *w32 = d == 0 ? wx32 : (d == 1 ? wy32 : wz32);
    w32[pa] = (float)w;
    unsigned int *word = (unsigned int *)(code + (pa & ~3ll));
    atomicOr(word, (unsigned int)(2u << d) << (8 * (pa & 3)));
}

// diag = ((((((Wx- + Wx+) + Wy-) + Wy+) + Wz-) + Wz+) + kappa), 0 on boundary.
__global__ void k_diag(const double *__restrict__ Wx, const double *__restrict__ Wy,
                       const double *__restrict__ Wz, const uint8_t *__restrict__ inside,
                       GridGeo g, double kap_s, double *__restrict__ diag) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    if (is_bnd(g, i, j, k)) {
        diag[a] = 0.0;
        return;
    }
    long long sy = g.nx, sz = (long long)g.nx * g.ny;
    double s = 0.0;
    s = s + Wx[a - 1];
    s = s + Wx[a];
    s = s + Wy[a - sy];
    s = s + Wy[a];
    s = s + Wz[a - sz];
    s = s + Wz[a];
    diag[a] = s + (inside[a] ? 0.0 : kap_s);
}

__global__ void k_kappa(const uint8_t *__restrict__ inside, long long N, double kap_s,
                        double *__restrict__ out) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a < N) out[a] = inside[a] ? 0.0 : kap_s;
}

// Trilinear cell and weights of atom j (cell = clamp(floor((x-o)/h), 0, n-2)).
struct Tri {
    long long c[3];
    double w[3][2];
};

__device__ __forceinline__ Tri tri_cell(const GridGeo &g, double x, double y, double z) {
    Tri t;
    double p[3] = {x, y, z};
    long long nn[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) {
        double u = (p[d] - g.o[d]) / g.h;
        long long c = (long long)floor(u);
        c = c < 0 ? 0 : (c > nn[d] - 2 ? nn[d] - 2 : c);
        double tt = u - (double)c;
        t.c[d] = c;
        t.w[d][0] = 1.0 - tt;
        t.w[d][1] = tt;
    }
    return t;
}

// One thread per (atom, corner).  The contributions to a node are summed in
// increasing atom order, starting from 0, by the thread of the smallest atom
// id touching that node -- the same order as a sequential loop over atoms, so
// the result is deterministic and independent of scheduling.
__global__ void k_deposit(const double *__restrict__ atoms, long long na, GridGeo g,
                          CellList cl, const int *__restrict__ cstart,
                          const int *__restrict__ clist, double coef0,
                          double *__restrict__ f) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 8 * na) return;
    long long i = t >> 3;
    int corner = (int)(t & 7);
    const double *X = atoms, *Y = atoms + na, *Z = atoms + 2 * na, *Q = atoms + 4 * na;
    Tri ti = tri_cell(g, X[i], Y[i], Z[i]);
    long long node[3] = {ti.c[0] + (corner & 1), ti.c[1] + ((corner >> 1) & 1),
                         ti.c[2] + ((corner >> 2) & 1)};
    // position of the node, cell of the node in the atom cell list
    double xa[3];
    int cc[3];
    for (int d = 0; d < 3; ++d) {
        xa[d] = g.o[d] + (double)node[d] * g.h;
        double u = floor((xa[d] - cl.lo[d]) / cl.cs);
        cc[d] = (u < -4.0) ? -4 : ((u > (double)cl.dim[d] + 4.0) ? cl.dim[d] + 4 : (int)u);
    }
    // collect atoms whose cell has this node as a corner, in id order
    constexpr int MAXC = 32;
    int ids[MAXC];
    int m = 0;
    for (int cz = cc[2] - 1; cz <= cc[2] + 1; ++cz) {
        if (cz < 0 || cz >= cl.dim[2]) continue;
        for (int cy = cc[1] - 1; cy <= cc[1] + 1; ++cy) {
            if (cy < 0 || cy >= cl.dim[1]) continue;
            for (int cx = cc[0] - 1; cx <= cc[0] + 1; ++cx) {
                if (cx < 0 || cx >= cl.dim[0]) continue;
                int cid = (cz * cl.dim[1] + cy) * cl.dim[0] + cx;
                for (int s = cstart[cid]; s < cstart[cid + 1]; ++s) {
                    int j = clist[s];
                    Tri tj = (j == i) ? ti : tri_cell(g, X[j], Y[j], Z[j]);
                    bool corner_of = true;
                    for (int d = 0; d < 3; ++d) {
                        long long off = node[d] - tj.c[d];
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
    if (m == 0 || ids[0] != (int)i) return;  // another thread owns this node
    double acc = 0.0;
    for (int q = 0; q < m; ++q) {
        int j = ids[q];
        Tri tj = (j == i) ? ti : tri_cell(g, X[j], Y[j], Z[j]);
        int dx = (int)(node[0] - tj.c[0]), dy = (int)(node[1] - tj.c[1]),
            dz = (int)(node[2] - tj.c[2]);
        double coef = coef0 * Q[j];
        acc += coef * (tj.w[0][dx] * tj.w[1][dy] * tj.w[2][dz]);
    }
    f[(node[2] * g.ny + node[1]) * g.nx + node[0]] = acc;
}

// f[a] += W_e phi_b for edges to Dirichlet nodes, in the order -x,+x,-y,+y,-z,+z.
__global__ void k_lift(const double *__restrict__ Wx, const double *__restrict__ Wy,
                       const double *__restrict__ Wz, const double *__restrict__ bc, GridGeo g,
                       double *__restrict__ f) {
    long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    if (is_bnd(g, i, j, k)) return;
    if (!(i == 1 || j == 1 || k == 1 || i == g.nx - 2 || j == g.ny - 2 || k == g.nz - 2)) return;
    const double *W[3] = {Wx, Wy, Wz};
    long long st[3] = {1, g.nx, (long long)g.nx * g.ny};
    long long c[3] = {i, j, k};
    long long n[3] = {g.nx, g.ny, g.nz};
    double v = f[a];
    for (int d = 0; d < 3; ++d) {
        if (c[d] - 1 == 0) v += W[d][a - st[d]] * bc[a - st[d]];
        if (c[d] + 1 == n[d] - 1) v += W[d][a] * bc[a + st[d]];
    }
    f[a] = v;
}

}  // namespace

pb_status assemble(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    const GridGeo &geo = g->geo;
    const long long N = geo.N;
    PadGeo &p = sys->pad;
    p.nx = geo.nx;
    p.ny = geo.ny;
    p.nz = geo.nz;
    p.sx = (geo.nx + 15) & ~15;  // 16 elements: TMA strides and code rows need 16 B
    p.sxy = (long long)p.sx * geo.ny;
    p.Np = p.sxy * geo.nz;
    p.N = N;
    for (int d = 0; d < 3; ++d) sys->W[d] = (double *)dalloc(sizeof(double) * N, s);
    sys->diag = (double *)dalloc(sizeof(double) * N, s);
    sys->rhs = (double *)dalloc(sizeof(double) * N, s);
    sys->bc = (double *)dalloc(sizeof(double) * N, s);
    sys->phi = (double *)dalloc(sizeof(double) * N, s);
    sys->code = (uint8_t *)dalloc((size_t)((p.Np + 15) & ~15ll), s);
    for (int d = 0; d < 3; ++d) sys->w32[d] = (float *)dalloc(sizeof(float) * p.Np, s);
    if (!sys->W[0] || !sys->W[1] || !sys->W[2] || !sys->diag || !sys->rhs || !sys->bc ||
        !sys->phi || !sys->code || !sys->w32[0] || !sys->w32[1] || !sys->w32[2])
        return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(sys->code, 0, (size_t)((p.Np + 15) & ~15ll), s));
    PB_CUDA_TRY(cudaMemsetAsync(sys->bc, 0, sizeof(double) * N, s));
    const double eps_in = sys->p.eps_in, eps_out = sys->p.eps_out, h = geo.h;
    k_coef_pure<<<cdiv(N, 256), 256, 0, s>>>(g->inside, geo, p, eps_in * h, eps_out * h, sys->W[0],
                                             sys->W[1], sys->W[2], sys->code);
    PB_LAUNCH_CHECK();
    if (g->ncross > 0) {
        k_coef_special<<<cdiv(g->ncross, 256), 256, 0, s>>>(g->cid, g->calpha, g->ncross, geo, p,
                                                            eps_in, eps_out, sys->W[0], sys->W[1],
                                                            sys->W[2], sys->w32[0], sys->w32[1],
                                                            sys->w32[2], sys->code);
        PB_LAUNCH_CHECK();
    }
    k_diag<<<cdiv(N, 256), 256, 0, s>>>(sys->W[0], sys->W[1], sys->W[2], g->inside, geo,
                                        sys->kap_s, sys->diag);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

pb_status deposit_rhs(pb_system *sys, cudaStream_t s) {
    pb_grid *g = sys->g;
    const GridGeo &geo = g->geo;
    PB_CUDA_TRY(cudaMemsetAsync(sys->rhs, 0, sizeof(double) * geo.N, s));
    double coef0 = 4.0 * M_PI * sys->lB;
    if (g->na > 0) {
        k_deposit<<<cdiv(8 * g->na, 128), 128, 0, s>>>(g->atoms, g->na, geo, g->cells,
                                                       g->cells.start, g->cells.atom, coef0,
                                                       sys->rhs);
        PB_LAUNCH_CHECK();
    }
    k_lift<<<cdiv(geo.N, 256), 256, 0, s>>>(sys->W[0], sys->W[1], sys->W[2], sys->bc, geo,
                                           sys->rhs);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

pb_status fill_kappa(const pb_system *sys, double *dst, cudaStream_t s) {
    k_kappa<<<cdiv(sys->g->geo.N, 256), 256, 0, s>>>(sys->g->inside, sys->g->geo.N, sys->kap_s,
                                                     dst);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

}  // namespace pbg
