// Krylov solve of the condensed system A phi = f (Sec. 3.1, Eq.
// matrixequation): Jacobi-preconditioned conjugate gradient with fused
// stencil/dot/axpy kernels, in FP64, or in FP32 inside FP64 iterative
// refinement.
//
// Iteration (z = D^-1 r is stored instead of r; r = D z is formed on the fly):
//   kernel P:  p <- z + beta p ;  q = A p ;  sigma = p.q      -> alpha = rho/sigma
//   kernel U:  q = A p (recomputed) ; x += alpha p ; z -= alpha D^-1 q ;
//              rho' = (Dz).z ; rr = |Dz|^2                    -> beta = rho'/rho
// Each kernel marches a tile of 32*VEC x TY nodes along z, keeping the p
// values of three planes in registers and one plane (plus the y halo rows,
// computed by two extra warps) in shared memory; x neighbours come from warp
// shuffles and one extra load at each tile edge.  Every global vector access
// is a 16-byte vector access on rows padded to a multiple of 4 elements.
// Dot products are accumulated per thread in the working precision and
// reduced across the grid in FP64 with a fixed order (last-block pattern),
// so results are deterministic.
//
// FP32 operator: per node one code byte (bit 0 solute, bits 1..3 "the +x/+y/+z
// edge is listed"); unlisted edges have the pure weight eps h of the node's
// medium, listed edges read their FP32 weight from the crossing list, found by
// a binary search inside the edge's row.  The diagonal is rebuilt from the
// six weights and the node's ionic term, so no coefficient array is streamed.
#include <math.h>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>
#include <type_traits>

#include "pb_internal.h"

namespace pbg {

namespace {

template <typename T>
struct VT;
template <>
struct VT<float> {
    using V = float4;
    static constexpr int N = 4;
};
template <>
struct VT<double> {
    using V = double2;
    static constexpr int N = 2;
};

template <typename T>
__device__ __forceinline__ void vload(const T *p, T (&v)[VT<T>::N]);
template <>
__device__ __forceinline__ void vload<float>(const float *p, float (&v)[4]) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
template <>
__device__ __forceinline__ void vload<double>(const double *p, double (&v)[2]) {
    double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x;
    v[1] = t.y;
}
template <typename T>
__device__ __forceinline__ void vstore(T *p, const T (&v)[VT<T>::N]);
template <>
__device__ __forceinline__ void vstore<float>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void vstore<double>(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

template <int VEC>
__device__ __forceinline__ uint32_t cload(const uint8_t *p);
template <>
__device__ __forceinline__ uint32_t cload<4>(const uint8_t *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}
template <>
__device__ __forceinline__ uint32_t cload<2>(const uint8_t *p) {
    return (uint32_t) * reinterpret_cast<const uint16_t *>(p);
}

// ------------------------------------------------------ operator providers --
// Compressed FP32 operator: weights of unlisted edges are the pure medium
// value of the node's code byte; a listed edge reads its FP32 weight from
// the padded per-node arrays wx/wy/wz, which are touched only for listed
// edges (a few percent of faces), so they are not streamed.
struct CoefC32 {
    static constexpr bool kCompressed = true;
    const float *wx, *wy, *wz;
    float w_in, w_out, kap;
    // weight of the edge along d whose low node has padded index pl and
    // code cl; cs is the code of the node being updated
    __device__ __forceinline__ float w(int d, int, int, int, int pl, uint8_t cl, uint8_t cs) const {
        const float *W = d == 0 ? wx : (d == 1 ? wy : wz);
        return ((cl >> (1 + d)) & 1) ? __ldg(W + pl) : ((cs & 1) ? w_in : w_out);
    }
    __device__ __forceinline__ float pure(uint8_t cs) const { return (cs & 1) ? w_in : w_out; }
    __device__ __forceinline__ float kappa(uint8_t cs) const { return (cs & 1) ? 0.f : kap; }
};

// Stored FP64 weights (canonical layout): the plain FP64 solver and the
// FP64 apply stream the three weight arrays.
struct CoefS64 {
    static constexpr bool kCompressed = false;
    const double *W0, *W1, *W2;
    double kap;
    int nx, ny;
    __device__ __forceinline__ double w(int d, int i, int j, int k, int, uint8_t, uint8_t) const {
        int a = (k * ny + j) * nx + i;
        return d == 0 ? W0[a] : (d == 1 ? W1[a] : W2[a]);
    }
    __device__ __forceinline__ double pure(uint8_t) const { return 0.0; }
    __device__ __forceinline__ double kappa(uint8_t cs) const { return (cs & 1) ? 0.0 : kap; }
};

enum { MODE_P = 0, MODE_U = 1, MODE_A = 2 };

template <typename T>
struct KArgs {
    const T *in;     // P: z ; U: p ; A: x
    const T *in2;    // P: p_old
    T *out;          // P: p_new ; A: y
    T *xv;           // U: x (solution increment)
    T *zv;           // U: z
    const uint8_t *code;
    CgState *st;
    double *partials;
    PadGeo pg;
    int KC;
    unsigned int *queue;  // TMA kernels: [0] next work item, [1] blocks finished
};

// block-wide FP64 sum of v (valid in thread 0)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sred) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sred[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NT / 32; ++q) t += sred[q];
    __syncthreads();
    return t;
}

// Sum partials[0..nb) (and partials[nb..2nb) when TWO) in a fixed order by the
// last block to finish; returns true in that block (all threads).  With
// REDUCED the block's own totals are already in thread 0's mine0/mine1.
template <int NT, bool TWO, bool REDUCED = false>
__device__ bool last_block_total(CgState *st, double *partials, int nb, double mine0,
                                 double mine1, double *sred, double &tot0, double &tot1) {
    __shared__ int s_last;
    int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double b0 = REDUCED ? mine0 : block_sum<NT>(mine0, sred);
    double b1 = TWO ? (REDUCED ? mine1 : block_sum<NT>(mine1, sred)) : 0.0;
    if (threadIdx.x == 0) {
        partials[bid] = b0;
        if (TWO) partials[nb + bid] = b1;
        __threadfence();
        unsigned t = atomicAdd(&st->counter, 1u);
        s_last = (t == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double a0 = 0.0, a1 = 0.0;
    for (int q = threadIdx.x; q < nb; q += NT) {
        a0 += __ldcg(partials + q);
        if (TWO) a1 += __ldcg(partials + nb + q);
    }
    tot0 = block_sum<NT>(a0, sred);
    tot1 = TWO ? block_sum<NT>(a1, sred) : 0.0;
    return true;
}

template <typename T>
__device__ __forceinline__ void sstore(T *dst, const T (&v)[VT<T>::N]) {
    vstore<T>(dst, v);
}

// code bytes of a lane's VEC points packed in one word
template <int VEC>
struct CodeW;
template <>
struct CodeW<4> {
    using W = uint32_t;
    static constexpr uint32_t rep(uint32_t b) { return b * 0x01010101u; }
};
template <>
struct CodeW<2> {
    using W = uint32_t;
    static constexpr uint32_t rep(uint32_t b) { return b * 0x0101u; }
};

// One stencil kernel for the three uses (MODE_P / MODE_U / MODE_A).
// Each warp owns one grid row j (32*VEC consecutive x nodes, VEC per lane)
// and marches along z over KC planes, carrying its row of planes k-1, k, k+1
// in registers; the rows j-1 and j+1 of plane k are read from L1/L2 (the
// neighbouring warps streamed them from HBM moments earlier), x neighbours
// come from warp shuffles plus one scalar load at each tile edge.  Warps
// never wait on each other; a block only synchronises for its final
// reduction.
template <typename T, class CP, int MODE, int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB)
k_stencil(KArgs<T> A, CP cp) {
    constexpr int VEC = VT<T>::N;
    constexpr int NT = 32 * WARPS;
    constexpr int TXP = 32 * VEC;
    __shared__ double sred[NT / 32];

    T alpha = 0, beta = 0;
    if (MODE != MODE_A) {
        if (A.st->done) return;
        if (MODE == MODE_P) beta = (T)A.st->beta;
        if (MODE == MODE_U) alpha = (T)A.st->alpha;
    }
    const PadGeo g = A.pg;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * TXP;
    const int ib = i0 + lane * VEC;  // first point of this lane
    const int j = 1 + blockIdx.y * WARPS + w;
    const int k0 = 1 + blockIdx.z * A.KC;
    const int k1 = min(k0 + A.KC, g.nz - 1);
    const bool active = j <= g.ny - 2;
    const bool grp_ok = active && ib < g.sx;
    const bool hl = active && lane == 0 && i0 > 0;
    const bool hr = active && lane == 31 && i0 + TXP < g.sx;
    const int sx = g.sx, sxy = (int)g.sxy;

    // streamed value at padded index q0 (P mode forms z + beta p_old)
    auto ldv = [&](int q0, T (&v)[VEC]) {
        vload<T>(A.in + q0, v);
        if (MODE == MODE_P) {
            T po[VEC];
            vload<T>(A.in2 + q0, po);
#pragma unroll
            for (int q = 0; q < VEC; ++q) v[q] = v[q] + beta * po[q];
        }
    };
    auto lds = [&](int q0) -> T {
        T v = A.in[q0];
        if (MODE == MODE_P) v = v + beta * A.in2[q0];
        return v;
    };

    // Software pipeline.  Entering iteration k (output plane k) registers
    // hold: own row at planes k-1, k, k+1 (pm, pc, pn); neighbour rows j-1,
    // j+1 at plane k (ym, yp); x and z at plane k (U mode).  Iteration k
    // issues the loads of plane k+2 (own row, raw) and plane k+1 (neighbour
    // rows, x, z) before computing plane k, so every load has a full
    // iteration to arrive.
    T pm[VEC], pc[VEC], pn[VEC];
    T ym[VEC], yp[VEC], xv[VEC], zv[VEC];
    uint32_t cm = 0, cc = 0, cn = 0, cym = 0;
    T lc = 0, rc = 0, ln = 0, rn = 0;
    uint32_t lcc = 0, lcn = 0;
#pragma unroll
    for (int q = 0; q < VEC; ++q) pm[q] = pc[q] = pn[q] = ym[q] = yp[q] = xv[q] = zv[q] = 0;
    if (grp_ok) {
        const int b0 = (k0 - 1) * sxy + j * sx + ib;
        ldv(b0, pm);
        cm = cload<VEC>(A.code + b0);
        ldv(b0 + sxy, pc);
        cc = cload<VEC>(A.code + b0 + sxy);
        ldv(b0 + 2 * sxy, pn);
        cn = cload<VEC>(A.code + b0 + 2 * sxy);
        ldv(b0 + sxy - sx, ym);
        ldv(b0 + sxy + sx, yp);
        cym = cload<VEC>(A.code + b0 + sxy - sx);
        if (MODE == MODE_U) {
            vload<T>(A.xv + b0 + sxy, xv);
            vload<T>(A.zv + b0 + sxy, zv);
        }
    }
    if (hl) {
        const int q0 = k0 * sxy + j * sx + i0 - 1;
        lc = lds(q0);
        lcc = A.code[q0];
        ln = lds(q0 + sxy);
        lcn = A.code[q0 + sxy];
    }
    if (hr) {
        const int q0 = k0 * sxy + j * sx + i0 + TXP;
        rc = lds(q0);
        rn = lds(q0 + sxy);
    }

    // fast-path diagonals of the two pure media and their inverses
    T dg_in = 1, dg_out = 1, dinv_in = 1, dinv_out = 1;
    if (CP::kCompressed) {
        dg_in = (T)6 * cp.pure(1) + cp.kappa(1);
        dg_out = (T)6 * cp.pure(0) + cp.kappa(0);
        dinv_in = (T)1 / dg_in;
        dinv_out = (T)1 / dg_out;
    }
    T acc0 = 0, acc1 = 0;

    for (int k = k0; k < k1; ++k) {
        const int base = k * sxy + j * sx;  // row j, plane k
        const bool more = k + 1 < k1;
        // ---- issue next loads
        T n2a[VEC], n2b[VEC];  // own row, plane k+2 (raw: z and p_old in P mode)
        T ymn[VEC], ypn[VEC], xvn[VEC], zvn[VEC];
        uint32_t cn2 = 0, cymn = 0;
        T ln2a = 0, ln2b = 0, rn2a = 0, rn2b = 0;
        uint32_t lcn2 = 0;
        if (grp_ok && more) {
            const int q2 = base + 2 * sxy + ib;
            vload<T>(A.in + q2, n2a);
            if (MODE == MODE_P) vload<T>(A.in2 + q2, n2b);
            cn2 = cload<VEC>(A.code + q2);
            ldv(base + sxy - sx + ib, ymn);
            ldv(base + sxy + sx + ib, ypn);
            cymn = cload<VEC>(A.code + base + sxy - sx + ib);
            if (MODE == MODE_U) {
                vload<T>(A.xv + base + sxy + ib, xvn);
                vload<T>(A.zv + base + sxy + ib, zvn);
            }
        }
        if (hl && more) {
            const int q2 = base + 2 * sxy + i0 - 1;
            ln2a = A.in[q2];
            if (MODE == MODE_P) ln2b = A.in2[q2];
            lcn2 = A.code[q2];
        }
        if (hr && more) {
            const int q2 = base + 2 * sxy + i0 + TXP;
            rn2a = A.in[q2];
            if (MODE == MODE_P) rn2b = A.in2[q2];
        }

        // ---- compute plane k
        T left = __shfl_up_sync(0xffffffffu, pc[VEC - 1], 1);
        T right = __shfl_down_sync(0xffffffffu, pc[0], 1);
        uint32_t lcode = __shfl_up_sync(0xffffffffu, cc >> (8 * (VEC - 1)), 1) & 0xffu;
        if (lane == 0) {
            left = lc;
            lcode = lcc;
        }
        if (lane == 31) right = rc;
        // code bytes of the -x neighbours of the lane's points
        const uint32_t cxl = (VEC == 4) ? ((cc << 8) | lcode) : (((cc << 8) | lcode) & 0xffffu);
        bool fast = false;
        if (CP::kCompressed) {
            const uint32_t special = (cc & CodeW<VEC>::rep(0x0Eu)) | (cxl & CodeW<VEC>::rep(0x02u)) |
                                     (cym & CodeW<VEC>::rep(0x04u)) | (cm & CodeW<VEC>::rep(0x08u));
            fast = !__any_sync(0xffffffffu, special != 0u);
        }
        T y[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            const int i = ib + q;
            const uint8_t c0 = (uint8_t)(cc >> (8 * q));
            const T x0 = pc[q];
            const T xl = q > 0 ? pc[q - 1] : left;
            const T xr = q < VEC - 1 ? pc[q + 1] : right;
            const T kp = cp.kappa(c0);
            T ap, dinv, dg;
            if (fast) {
                const T wp = cp.pure(c0);
                const T sum = ((x0 - xl) + (x0 - xr)) + ((x0 - ym[q]) + (x0 - yp[q])) +
                              ((x0 - pm[q]) + (x0 - pn[q]));
                ap = wp * sum + kp * x0;
                dinv = (c0 & 1) ? dinv_in : dinv_out;
                dg = (c0 & 1) ? dg_in : dg_out;
            } else {
                const int pl = base + i;
                const T wxp = cp.w(0, i, j, k, pl, c0, c0);
                const T wxm = cp.w(0, i - 1, j, k, pl - 1, (uint8_t)(cxl >> (8 * q)), c0);
                const T wyp = cp.w(1, i, j, k, pl, c0, c0);
                const T wym = cp.w(1, i, j - 1, k, pl - sx, (uint8_t)(cym >> (8 * q)), c0);
                const T wzp = cp.w(2, i, j, k, pl, c0, c0);
                const T wzm = cp.w(2, i, j, k - 1, pl - sxy, (uint8_t)(cm >> (8 * q)), c0);
                ap = kp * x0;
                ap += wxm * (x0 - xl);
                ap += wxp * (x0 - xr);
                ap += wym * (x0 - ym[q]);
                ap += wyp * (x0 - yp[q]);
                ap += wzm * (x0 - pm[q]);
                ap += wzp * (x0 - pn[q]);
                dg = ((((((wxm + wxp) + wym) + wyp) + wzm) + wzp) + kp);
                dinv = (T)1 / dg;
            }
            const bool interior = grp_ok && i >= 1 && i <= g.nx - 2;
            y[q] = interior ? ap : (T)0;
            if (MODE == MODE_P) {
                if (interior) acc0 += x0 * ap;
            } else if (MODE == MODE_U) {
                if (interior) {
                    xv[q] = xv[q] + alpha * x0;
                    const T znew = zv[q] - alpha * ap * dinv;
                    zv[q] = znew;
                    const T r = dg * znew;
                    acc0 += r * znew;
                    acc1 += r * r;
                }
            }
        }
        if (grp_ok) {
            if (MODE == MODE_P) vstore<T>(A.out + base + ib, pc);
            if (MODE == MODE_U) {
                vstore<T>(A.xv + base + ib, xv);
                vstore<T>(A.zv + base + ib, zv);
            }
            if (MODE == MODE_A) vstore<T>(A.out + base + ib, y);
        }
        // ---- rotate the pipeline
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
            pm[q] = pc[q];
            pc[q] = pn[q];
            pn[q] = (MODE == MODE_P) ? n2a[q] + beta * n2b[q] : n2a[q];
            ym[q] = ymn[q];
            yp[q] = ypn[q];
            if (MODE == MODE_U) {
                xv[q] = xvn[q];
                zv[q] = zvn[q];
            }
        }
        cm = cc;
        cc = cn;
        cn = cn2;
        cym = cymn;
        lc = ln;
        rc = rn;
        lcc = lcn;
        ln = (MODE == MODE_P) ? ln2a + beta * ln2b : ln2a;
        rn = (MODE == MODE_P) ? rn2a + beta * rn2b : rn2a;
        lcn = lcn2;
    }
    if (MODE == MODE_A) return;

    const int nb = gridDim.x * gridDim.y * gridDim.z;
    double t0, t1;
    if (MODE == MODE_P) {
        if (last_block_total<NT, false>(A.st, A.partials, nb, (double)acc0, 0.0, sred, t0, t1)) {
            if (threadIdx.x == 0) {
                CgState *s = A.st;
                s->sigma = t0;
                if (s->profile) {
                    s->alpha = isfinite(t0) && t0 != 0.0 ? s->rho / t0 : 0.0;
                } else if (!(t0 > 0.0) || !isfinite(t0)) {
                    s->done = 1;
                    s->status = 1;
                } else {
                    s->alpha = s->rho / t0;
                }
                s->counter = 0;
            }
        }
    } else {
        if (last_block_total<NT, true>(A.st, A.partials, nb, (double)acc0, (double)acc1, sred, t0,
                                       t1)) {
            if (threadIdx.x == 0) {
                CgState *s = A.st;
                s->beta = t0 / s->rho;
                s->rho = t0;
                s->rr = t1;
                s->iter += 1;
                if (s->profile) {
                    // timing run: keep going
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
                s->counter = 0;
            }
        }
    }
}

#include "stencil_tma.cuh"
#include "cg64.cuh"

// FP64 true residual r = f - A phi on interior nodes (boundary neighbours
// read their Dirichlet value through the lift already in f, so they are
// masked here).  Writes z = r/diag to the padded solver layout (FP32 or FP64),
// and r itself when rout is given (the plain FP64 solver keeps r), and
// reduces |r|^2 and r.z.  Persistent grid (the blocks resident on the
// GPU): the stencil is the only FP64 arithmetic per node; for the FP32 solver
// |r|^2 and r.z are summed in FP32 per thread and per block (they serve as
// stopping norms and as the restart rho of the FP32 PCG) and in FP64 across
// blocks, in a fixed order.
template <typename TZ>
__global__ void __launch_bounds__(256)
k_residual(const double *__restrict__ phi, const double *__restrict__ f,
           const double *__restrict__ Wx, const double *__restrict__ Wy,
           const double *__restrict__ Wz, const double *__restrict__ diag, GridGeo g, PadGeo pg,
           TZ *__restrict__ zout, CgState *st, double *partials, double *__restrict__ rout,
           int kofs = 0, int nzg = 0) {
    __shared__ double sred[8];
    __shared__ TZ sblk[2][8];
    const long long stride = (long long)gridDim.x * 256;
    const bool narrow = g.N <= 0x7fffffffll;
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    TZ rr = 0, rz = 0;
    for (long long a = blockIdx.x * 256ll + threadIdx.x; a < g.N; a += stride) {
        long long i, j, k;
        if (narrow) {
            unsigned ua = (unsigned)a, row = ua / (unsigned)g.nx;
            i = ua - row * (unsigned)g.nx;
            j = row % (unsigned)g.ny;
            k = row / (unsigned)g.ny;
        } else {
            i = a % g.nx;
            j = (a / g.nx) % g.ny;
            k = a / sz;
        }
        bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
        if (!interior) continue;
        double x0 = phi[a];
        double sum = diag[a] * x0;
        if (i > 1) sum -= Wx[a - 1] * phi[a - 1];
        if (i < g.nx - 2) sum -= Wx[a] * phi[a + 1];
        if (j > 1) sum -= Wy[a - sy] * phi[a - sy];
        if (j < g.ny - 2) sum -= Wy[a] * phi[a + sy];
        // a slab of a split solve: local plane k is global plane k + kofs
        if (k + kofs > 1) sum -= Wz[a - sz] * phi[a - sz];
        if (k + kofs < (nzg > 0 ? nzg : g.nz) - 2) sum -= Wz[a] * phi[a + sz];
        double r = f[a] - sum;
        TZ z, rt;
        if (sizeof(TZ) == 4) {
            rt = (TZ)(float)r;
            z = (TZ)((float)r / (float)diag[a]);
        } else {
            rt = (TZ)r;
            z = (TZ)(r / diag[a]);
        }
        zout[(k * g.ny + j) * pg.sx + i] = z;
        if (rout) rout[(k * g.ny + j) * pg.sx + i] = r;
        rr += rt * rt;
        rz += rt * z;
    }
    // block sums in the accumulation type, then FP64 across blocks
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        rz += __shfl_down_sync(0xffffffffu, rz, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sblk[0][threadIdx.x >> 5] = rr;
        sblk[1][threadIdx.x >> 5] = rz;
    }
    __syncthreads();
    double b0 = 0.0, b1 = 0.0;
    if (threadIdx.x == 0) {
        TZ t0 = 0, t1 = 0;
        for (int q = 0; q < 8; ++q) {
            t0 += sblk[0][q];
            t1 += sblk[1][q];
        }
        b0 = (double)t0;
        b1 = (double)t1;
    }
    int nb = gridDim.x;
    double t0, t1;
    if (last_block_total<256, true, true>(st, partials, nb, b0, b1, sred, t0, t1)) {
        if (threadIdx.x == 0) {
            st->res64 = t0;
            st->rz64 = t1;
            st->counter = 0;
        }
    }
}

// phi(interior) += x (padded)
template <typename TX>
__global__ void k_promote(double *__restrict__ phi, const TX *__restrict__ x, GridGeo g, PadGeo pg) {
    long long a = blockIdx.x * 256ll + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
    if (interior) phi[a] += (double)x[(k * g.ny + j) * pg.sx + i];
}

template <typename T>
__global__ void k_canon_to_pad(const T *__restrict__ src, T *__restrict__ dst, GridGeo g, PadGeo pg) {
    long long a = blockIdx.x * 256ll + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
    dst[(k * g.ny + j) * pg.sx + i] = interior ? src[a] : (T)0;
}

template <typename T>
__global__ void k_pad_to_canon(const T *__restrict__ src, T *__restrict__ dst, GridGeo g, PadGeo pg) {
    long long a = blockIdx.x * 256ll + threadIdx.x;
    if (a >= g.N) return;
    long long i = a % g.nx, j = (a / g.nx) % g.ny, k = a / ((long long)g.nx * g.ny);
    bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
    dst[a] = interior ? src[(k * g.ny + j) * pg.sx + i] : (T)0;
}

constexpr int TYC = 8;  // rows (warps) per stencil block
// resident blocks per SM the register allocation must allow
template <typename T>
struct MinB {
    static constexpr int v = sizeof(T) == 4 ? 3 : 2;
};

template <typename T>
dim3 stencil_grid(const PadGeo &g, int KC) {
    constexpr int TXP = 32 * VT<T>::N;
    return dim3((unsigned)cdiv(g.nx - 1, TXP), (unsigned)cdiv(g.ny - 2, TYC),
                (unsigned)cdiv(g.nz - 2, KC));
}

// z-chunk length: trade the two extra planes each chunk reads against the
// tail of the last wave (blocks resident per SM from the occupancy API).
template <typename T, class CP>
int choose_kc(const PadGeo &g) {
    static int resident = 0;
    if (!resident) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_stencil<T, CP, MODE_U, TYC, MinB<T>::v>, 32 * TYC, 0) != cudaSuccess ||
            per_sm <= 0) {
            cudaGetLastError();
            per_sm = MinB<T>::v;
        }
        resident = per_sm * num_sms();
    }
    long long cols = (long long)cdiv(g.nx - 1, 32 * VT<T>::N) * cdiv(g.ny - 2, TYC);
    int best = 8;
    double best_eff = -1.0;
    for (int kc = 4; kc <= 64; ++kc) {
        long long blocks = cols * cdiv(g.nz - 2, kc);
        double waves = (double)blocks / resident;
        double occ = waves / ceil(waves);
        double stream = (double)kc / (kc + 1.0);  // about half the streamed arrays re-read 2 planes
        double eff = occ * stream;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = kc;
        }
    }
    return best;
}

int default_kc(const PadGeo &g, int precision) {
    return precision == PB_MIXED ? choose_kc<float, CoefC32>(g) : choose_kc<double, CoefS64>(g);
}

// ------------------------------------------------------ TMA tensor maps --
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D tiled map over a padded (sx, ny, nz) array; box (bw, bh, 1)
pb_status make_map(CUtensorMap *m, const void *base, bool bytes, const PadGeo &g, int bw, int bh) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available");
        return PB_ERR_CUDA;
    }
    const uint64_t esz = bytes ? 1 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)g.sx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.sx * esz, (cuuint64_t)g.sxy * esz};
    cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return PB_ERR_CUDA;
    }
    return PB_OK;
}

// maps of one TMA stencil launch with tiles of width tw
pb_status tma_maps(const pb_system *sys, int mode, const float *a, const float *b, const float *x,
                   const float *z, tma::Maps *m, int tw) {
    const PadGeo &g = sys->pad;
    const int bw = tma::box_w(tw), bh = tma::box_h(tw), th = tma::tile_h(tw);
    pb_status rc = make_map(&m->a, a, false, g, bw, bh);
    if (rc == PB_OK && mode == MODE_P) rc = make_map(&m->b, b, false, g, bw, bh);
    if (rc == PB_OK && mode == MODE_U) rc = make_map(&m->x, x, false, g, tw, th);
    if (rc == PB_OK && mode == MODE_U) rc = make_map(&m->z, z, false, g, tw, th);
    if (rc == PB_OK) rc = make_map(&m->code, sys->code, true, g, tma::code_w(tw), bh);
    return rc;
}

template <int MODE>
pb_status tma_prepare() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_stencil_tma<MODE, false, 0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tma::smem_bytes<MODE, 0>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stencil_tma<MODE, true, 0>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tma::smem_bytes<MODE, 0>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stencil_tma<MODE, true, tma::TWDEF>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     tma::smem_bytes<MODE, tma::TWDEF>());
        if (e != cudaSuccess) {
            set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
            return PB_ERR_CUDA;
        }
        done = true;
    }
    return PB_OK;
}

// one block per resident slot (persistent, balanced ranges), at most one
// block per (tile column, plane) pair
dim3 tma_grid(const PadGeo &g, int) {
    static int per_sm = 0;
    if (!per_sm) {
        if (tma_prepare<MODE_U>() != PB_OK ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil_tma<MODE_U, false, 0>,
                                                          tma::NTHREADS,
                                                          tma::smem_bytes<MODE_U, 0>()) != cudaSuccess ||
            per_sm <= 0) {
            cudaGetLastError();
            per_sm = 2;
        }
    }
    return dim3((unsigned)std::max(per_sm * num_sms(), 1));
}

template <int MODE>
void tma_launch(const tma::SysEntry *dev_tab, int nsys, int total_items, unsigned int *queue,
                dim3 grid, cudaStream_t s, const tma::SysEntry *host_e0 = nullptr,
                bool overlap = false) {
    // host_e0: the host copy of the entry of a one-system launch, passed by
    // value (the single-system kernel reads everything of it from the
    // parameter bank); nullptr or several systems: the table form.
    // overlap: programmatic stream serialization, so that this launch's
    // blocks start (and set up) while the previous stencil kernel drains.
    static const tma::SysEntry zero{};
    // one-system launches on the default tile width take the kernel that
    // has it as a constant
    const bool fixw = host_e0 && nsys == 1 && host_e0->tw == tma::TWDEF;
    if (host_e0 && nsys == 1 && overlap) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(tma::NTHREADS);
        cfg.dynamicSmemBytes = fixw ? tma::smem_bytes<MODE, tma::TWDEF>() : tma::smem_bytes<MODE, 0>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (fixw)
            cudaLaunchKernelEx(&cfg, k_stencil_tma<MODE, true, tma::TWDEF>, dev_tab, nsys,
                               total_items, queue, *host_e0);
        else
            cudaLaunchKernelEx(&cfg, k_stencil_tma<MODE, true, 0>, dev_tab, nsys, total_items,
                               queue, *host_e0);
    } else if (fixw)
        k_stencil_tma<MODE, true, tma::TWDEF><<<grid, tma::NTHREADS, tma::smem_bytes<MODE, tma::TWDEF>(), s>>>(
            dev_tab, nsys, total_items, queue, *host_e0);
    else if (host_e0 && nsys == 1)
        k_stencil_tma<MODE, true, 0><<<grid, tma::NTHREADS, tma::smem_bytes<MODE, 0>(), s>>>(
            dev_tab, nsys, total_items, queue, *host_e0);
    else
        k_stencil_tma<MODE, false, 0><<<grid, tma::NTHREADS, tma::smem_bytes<MODE, 0>(), s>>>(
            dev_tab, nsys, total_items, queue, zero);
}

struct TmaState {
    tma::SysEntry host;          // this system's launch-table entry
    tma::SysEntry *dev = nullptr;  // device copy (a table of one)
    float *partials = nullptr;   // per-item dot-product slots
    unsigned int *cnt = nullptr;
    int tw = tma::TWDEF;         // tile width of the maps in host
    int uploaded_kc = -1, uploaded_tw = -1;
    int max_items = 0;
};

int tma_items(const PadGeo &g, int KC, int tw) {
    return (int)(cdiv(g.nx - 1, tw) * cdiv(g.ny - 2, tma::tile_h(tw)) * cdiv(g.nz - 2, KC));
}

// entry fields that depend on the z-chunk length and the tile width
void tma_entry_geometry(tma::SysEntry &e, const PadGeo &g, int KC, int tw) {
    e.tw = tw;
    e.xtiles = (int)cdiv(g.nx - 1, tw);
    e.ytiles = (int)cdiv(g.ny - 2, tma::tile_h(tw));
    e.KC = KC;
    e.nchunk = (int)cdiv(g.nz - 2, KC);
    e.nitems = e.xtiles * e.ytiles * e.nchunk;
    e.item_base = 0;
}

// the direction and update maps of a system's entry for tiles of width tw
pb_status tma_sys_maps(pb_system *sys, tma::SysEntry &e, int tw) {
    const float *pbuf[2] = {sys->pa32, sys->pb32};
    pb_status rc = PB_OK;
    for (int c = 0; c < 2 && rc == PB_OK; ++c) {
        rc = tma_maps(sys, MODE_P, sys->z32, pbuf[c], nullptr, nullptr, &e.P[c], tw);
        if (rc == PB_OK)
            rc = tma_maps(sys, MODE_U, pbuf[c ^ 1], nullptr, sys->d32, sys->z32, &e.U[c], tw);
    }
    return rc;
}

CoefC32 make_c32(const pb_system *sys);

pb_status build_tma_state(pb_system *sys) {
    if (sys->tma) return PB_OK;
    TmaState *t = new (std::nothrow) TmaState();
    if (!t) return PB_ERR_OOM;
    cudaStream_t s = sys->stream;
    pb_status rc = PB_OK;
    tma::SysEntry &e = t->host;
    rc = tma_sys_maps(sys, e, t->tw);
    e.tw = t->tw;
    if (rc == PB_OK) rc = tma_prepare<MODE_P>();
    if (rc == PB_OK) rc = tma_prepare<MODE_U>();
    if (rc == PB_OK) rc = tma_prepare<MODE_A>();
    e.pg = sys->pad;
    e.cp = make_c32(sys);
    e.pbuf[0] = sys->pa32;
    e.pbuf[1] = sys->pb32;
    e.x = sys->d32;
    e.z = sys->z32;
    e.y = nullptr;
    e.st = sys->st;
    t->max_items = std::max(tma_items(sys->pad, 4, 128),
                            std::max(tma_items(sys->pad, 4, 64), tma_items(sys->pad, 4, 32)));
    if (rc == PB_OK) {
        t->dev = (tma::SysEntry *)dalloc(sizeof(tma::SysEntry), s);
        t->partials = (float *)dalloc(sizeof(float) * 3 * (size_t)t->max_items, s);
        t->cnt = (unsigned int *)dalloc(4 * sizeof(unsigned int), s);
        if (!t->dev || !t->partials || !t->cnt) rc = PB_ERR_OOM;
    }
    if (rc == PB_OK && cudaMemsetAsync(t->cnt, 0, 4 * sizeof(unsigned int), s) != cudaSuccess)
        rc = PB_ERR_CUDA;
    if (rc != PB_OK) {
        dfree(t->dev, s);
        dfree(t->partials, s);
        dfree(t->cnt, s);
        delete t;
        return rc;
    }
    e.partials = t->partials;
    e.cnt = t->cnt;
    sys->tma = t;
    return PB_OK;
}

// make the host entry's maps those of tiles of width tw (host only)
pb_status tma_set_tile(pb_system *sys, int tw) {
    TmaState *t = (TmaState *)sys->tma;
    if (t->tw == tw) return PB_OK;
    pb_status rc = tma_sys_maps(sys, t->host, tw);
    if (rc != PB_OK) return rc;
    t->tw = tw;
    t->host.tw = tw;
    t->uploaded_kc = -1;
    return PB_OK;
}

// make the device entry describe z-chunks of KC planes (KC >= 4) of tiles
// of width tw
pb_status tma_use_kc(pb_system *sys, int KC, int tw, cudaStream_t s) {
    TmaState *t = (TmaState *)sys->tma;
    if (KC < 4) KC = 4;
    pb_status rc = tma_set_tile(sys, tw);
    if (rc != PB_OK) return rc;
    if (t->uploaded_kc == KC && t->uploaded_tw == tw) return PB_OK;
    tma_entry_geometry(t->host, sys->pad, KC, tw);
    PB_CUDA_TRY(cudaMemcpyAsync(t->dev, &t->host, sizeof(tma::SysEntry), cudaMemcpyHostToDevice, s));
    // the host copy must not change before the copy has been made
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    t->uploaded_kc = KC;
    t->uploaded_tw = tw;
    return PB_OK;
}

// one FP32 PCG iteration (direction + update kernels) with TMA staging;
// cur selects which of pa/pb holds p_old; blocks > 0 sets the grid size
// (timing runs), else one block per resident slot
void launch_iter_tma(pb_system *sys, const CoefC32 &, int cur, int KC, int tw, cudaStream_t s,
                     unsigned blocks = 0) {
    TmaState *t = (TmaState *)sys->tma;
    if (tma_use_kc(sys, KC, tw, s) != PB_OK) return;
    dim3 grid = blocks ? dim3(blocks) : tma_grid(sys->pad, KC);
    tma_launch<MODE_P>(t->dev, 1, t->host.nitems, sys->queue, grid, s, &t->host, true);
    tma_launch<MODE_U>(t->dev, 1, t->host.nitems, sys->queue, grid, s, &t->host, true);
}

CoefC32 make_c32(const pb_system *sys) {
    const pb_grid *g = sys->g;
    CoefC32 c;
    c.wx = sys->w32[0];
    c.wy = sys->w32[1];
    c.wz = sys->w32[2];
    c.w_in = (float)(sys->p.eps_in * g->geo.h);
    c.w_out = (float)(sys->p.eps_out * g->geo.h);
    c.kap = (float)sys->kap_s;
    return c;
}

CoefS64 make_s64(const pb_system *sys) {
    CoefS64 c;
    c.W0 = sys->W[0];
    c.W1 = sys->W[1];
    c.W2 = sys->W[2];
    c.kap = sys->kap_s;
    c.nx = sys->g->geo.nx;
    c.ny = sys->g->geo.ny;
    return c;
}

template <typename T, class CP>
pb_status launch_iter(pb_system *sys, const CP &cp, const T *z, const T *pold, T *pnew, T *x,
                      T *zmut, int KC, cudaStream_t s) {
    dim3 grid = stencil_grid<T>(sys->pad, KC);
    KArgs<T> a{};
    a.code = sys->code;
    a.st = sys->st;
    a.partials = sys->partials;
    a.pg = sys->pad;
    a.KC = KC;
    a.in = z;
    a.in2 = pold;
    a.out = pnew;
    k_stencil<T, CP, MODE_P, TYC, MinB<T>::v><<<grid, 32 * TYC, 0, s>>>(a, cp);
    KArgs<T> b = a;
    b.in = pnew;
    b.in2 = nullptr;
    b.out = nullptr;
    b.xv = x;
    b.zv = zmut;
    k_stencil<T, CP, MODE_U, TYC, MinB<T>::v><<<grid, 32 * TYC, 0, s>>>(b, cp);
    return PB_OK;
}

// one plain FP64 PCG iteration (direction + update kernels); cur selects
// which of pa/pb holds p_old; which: 0 direction only, 1 update only, 2 both
void launch_iter_cg64(pb_system *sys, int cur, int KC, cudaStream_t s, int which = 2) {
    const PadGeo &g = sys->pad;
    double *pbuf[2] = {sys->pa64, sys->pb64};
    cg64::DirArgs d{};
    d.z = sys->z64;
    d.pold = pbuf[cur];
    d.p = pbuf[cur ^ 1];
    d.q = sys->q64;
    d.w0 = sys->op64[0];
    d.w1 = sys->op64[1];
    d.w2 = sys->op64[2];
    d.dg = sys->op64[3];
    d.st = sys->st;
    d.partials = sys->partials;
    d.g = g;
    d.KC = KC;
    const dim3 grid((unsigned)cdiv(g.nx - 1, cg64::TXP), (unsigned)cdiv(g.ny - 2, cg64::WARPS),
                    (unsigned)cdiv(g.nz - 2, KC));
    if (which != 1) k_cg64_dir<<<grid, cg64::NT, 0, s>>>(d);
    if (which == 0) return;
    cg64::UpdArgs u{};
    u.x = sys->x64;
    u.r = sys->r64;
    u.z = sys->z64;
    u.p = pbuf[cur ^ 1];
    u.q = sys->q64;
    u.dinv = sys->op64[4];
    u.st = sys->st;
    u.partials = sys->partials;
    u.first = g.sxy;
    u.count = (long long)(g.nz - 2) * g.sxy;
    static int per_sm = 0;
    if (!per_sm &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg64_upd, cg64::UNT, 0) != cudaSuccess ||
         per_sm <= 0)) {
        cudaGetLastError();
        per_sm = 4;
    }
    // partials holds two slots per block
    const long long blocks = std::min<long long>(
        std::min<long long>(cdiv(u.count / 2, cg64::UNT), (long long)per_sm * num_sms()), sys->npartials / 2);
    k_cg64_upd<<<(unsigned)blocks, cg64::UNT, 0, s>>>(u);
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

pb_status sync_state(pb_system *sys, cudaStream_t s) {
    PB_CUDA_TRY(cudaMemcpyAsync(sys->h_st, sys->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return PB_OK;
}

// resident blocks of a 256-thread kernel on the whole GPU
template <class K>
long long resident_blocks(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 2;
    }
    return (long long)per_sm * num_sms();
}

pb_status residual(pb_system *sys, bool fp32_out, cudaStream_t s) {
    const GridGeo &g = sys->g->geo;
    static const long long res32 = resident_blocks(k_residual<float>);
    static const long long res64 = resident_blocks(k_residual<double>);
    unsigned blocks = (unsigned)std::min<long long>(cdiv(g.N, 256), fp32_out ? res32 : res64);
    if (fp32_out)
        k_residual<float><<<blocks, 256, 0, s>>>(sys->phi, sys->rhs, sys->W[0], sys->W[1], sys->W[2],
                                                 sys->diag, g, sys->pad, sys->z32, sys->st,
                                                 sys->partials, nullptr);
    else
        k_residual<double><<<blocks, 256, 0, s>>>(sys->phi, sys->rhs, sys->W[0], sys->W[1],
                                                  sys->W[2], sys->diag, g, sys->pad, sys->z64,
                                                  sys->st, sys->partials, sys->r64);
    PB_LAUNCH_CHECK();
    return PB_OK;
}

// Runs PCG iterations until the device state says done; host polls a pinned
// copy of the state after every chunk, keeping two chunks in flight.
template <typename T, class CP>
pb_status run_pcg(pb_system *sys, const CP &cp, T *z, T *pa, T *pb, T *x, int KC, int variant,
                  int tw, int chunk,
                  double deadline, cudaStream_t s, int *iters_out) {
    T *bufs[2] = {pa, pb};
    int cur = 0;  // index of p_old
    cudaEvent_t ev[2];
    PB_CUDA_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    PB_CUDA_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    CgState *hs = sys->h_st;  // two slots: hs[0], hs[1]
    pb_status rc = PB_OK;
    auto issue = [&](int slot) -> pb_status {
        for (int c = 0; c < chunk; ++c) {
            if constexpr (std::is_same<T, float>::value) {
                if (variant == 1)
                    launch_iter_tma(sys, cp, cur, KC, tw, s);
                else
                    launch_iter<T, CP>(sys, cp, z, bufs[cur], bufs[cur ^ 1], x, z, KC, s);
            } else {
                launch_iter_cg64(sys, cur, KC, s);
            }
            cur ^= 1;
        }
        note_launch(2 * chunk - 1);
        PB_LAUNCH_CHECK();
        PB_CUDA_TRY(cudaMemcpyAsync(hs + slot, sys->st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaEventRecord(ev[slot], s));
        return PB_OK;
    };
    int slot = 0;
    // every chunk advances the device iteration count by `chunk` unless the
    // state is done, so this many chunks always suffice
    long long max_chunks = (long long)hs[2].max_iter / chunk + 4;
    long long issued = 0;
    if ((rc = issue(0)) != PB_OK) goto out;
    if ((rc = issue(1)) != PB_OK) goto out;
    issued = 2;
    for (;;) {
        cudaError_t e = cudaEventSynchronize(ev[slot]);
        if (e != cudaSuccess) {
            set_error("PCG chunk failed: %s", cudaGetErrorString(e));
            rc = PB_ERR_CUDA;
            break;
        }
        if (hs[slot].done) break;
        if (deadline > 0.0 && now_s() > deadline) {
            rc = PB_ERR_TIMEOUT;
            break;
        }
        if (++issued > max_chunks) {
            set_error("PCG state stopped advancing");
            rc = PB_ERR_CUDA;
            break;
        }
        if ((rc = issue(slot)) != PB_OK) break;
        slot ^= 1;
    }
out:
    // drain and read the final state
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error("PCG failed: %s", cudaGetErrorString(e));
            rc = PB_ERR_CUDA;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc == PB_OK) {
        pb_status r2 = sync_state(sys, s);
        if (r2 != PB_OK) return r2;
        *iters_out = hs[0].iter;
    }
    return rc;
}

pb_status init_state(pb_system *sys, double rho, double rr0, double rr_stop, int max_iter,
                     cudaStream_t s, int profile = 0) {
    CgState h{};
    h.profile = profile;
    h.rho = rho;
    h.rr0 = rr0;
    h.rr = rr0;
    h.rr_stop = rr_stop;
    h.beta = 0.0;
    h.alpha = 0.0;
    h.iter = 0;
    h.max_iter = max_iter;
    h.done = 0;
    h.status = 0;
    h.counter = 0;
    // staged through the pinned mirror so the copy is stream-ordered
    CgState *stage = sys->h_st + 2;
    *stage = h;
    PB_CUDA_TRY(cudaMemcpyAsync(sys->st, stage, sizeof(CgState), cudaMemcpyHostToDevice, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return PB_OK;
}

// ---------------------------------------------------------------- tuner --
// Kernel variant (0: register-pipelined warps, 1: TMA-staged, FP32 only),
// z-chunk length and (TMA-staged) tile width chosen by timing PCG iterations
// of each candidate on the system itself; cached per (precision, grid shape).
struct Tuning {
    int variant = 0;
    int kc = 8;
    int tw = tma::TWDEF;
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, Tuning> g_tune;

// one PCG iteration of the given kernel variant, z-chunk and tile width
// (timing runs; blocks > 0: the TMA-staged kernels on that many blocks)
void tune_iter(pb_system *sys, int precision, int variant, int kc, int tw, int r, cudaStream_t s,
               unsigned blocks = 0) {
    if (precision == PB_MIXED) {
        CoefC32 cp = make_c32(sys);
        if (variant == 1)
            launch_iter_tma(sys, cp, r & 1, kc, tw, s, blocks);
        else
            launch_iter<float, CoefC32>(sys, cp, sys->z32, (r & 1) ? sys->pb32 : sys->pa32,
                                        (r & 1) ? sys->pa32 : sys->pb32, sys->d32, sys->z32, kc, s);
    } else {
        launch_iter_cg64(sys, r & 1, kc, s);
    }
    note_launch(2);
}

// time of two PCG iterations with z-chunk kc and tile width tw (after one
// untimed iteration, which also absorbs the switch of the launch-table entry);
// blocks > 0: the TMA-staged kernels on that many blocks
pb_status time_candidate(pb_system *sys, int precision, int variant, int kc, int tw,
                         cudaStream_t s, float *ms, unsigned blocks = 0) {
    cudaEvent_t ev[2];
    PB_CUDA_TRY(cudaEventCreate(&ev[0]));
    PB_CUDA_TRY(cudaEventCreate(&ev[1]));
    tune_iter(sys, precision, variant, kc, tw, 0, s, blocks);
    PB_CUDA_TRY(cudaEventRecord(ev[0], s));
    tune_iter(sys, precision, variant, kc, tw, 1, s, blocks);
    tune_iter(sys, precision, variant, kc, tw, 2, s, blocks);
    PB_CUDA_TRY(cudaEventRecord(ev[1], s));
    PB_CUDA_TRY(cudaEventSynchronize(ev[1]));
    PB_CUDA_TRY(cudaGetLastError());
    float t = 0.f;
    PB_CUDA_TRY(cudaEventElapsedTime(&t, ev[0], ev[1]));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    *ms = t / 2.0f;
    return PB_OK;
}

pb_status autotune(pb_system *sys, int precision, cudaStream_t s, Tuning *out) {
    const PadGeo &g = sys->pad;
    auto key = std::make_tuple(precision, g.nx, g.ny, g.nz);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *out = it->second;
            return PB_OK;
        }
    }
    // timing runs use the profile state (never stop); the solver re-initialises
    // every vector they touch before iterating
    pb_status rc = init_state(sys, 1.0, 1.0, -1.0, 1 << 30, s, 1);
    if (rc != PB_OK) return rc;
    // mixed precision always runs the TMA-staged kernels (the batched solver
    // shares them, so a system gives the same bits alone and in a batch);
    // their z-chunk and tile width are tuned.  FP64 runs the
    // register-pipelined kernels, whose z-chunk is tuned.
    const int variant = precision == PB_MIXED ? 1 : 0;
    Tuning best;
    best.variant = variant;
    const int kcs[] = {8, 6, 11, 16, 22, 32};  // first = default
    // tile widths: those whose tiles cover the interior of a plane with the
    // fewest idle lanes (smallest padded area), widest first.  A small grid
    // timed alone cannot fill the GPU, so its timings would not show the idle
    // lanes it costs when it shares launches with other systems (a 97-node
    // grid leaves a quarter of a 128-wide tile idle); the widths that tie are
    // timed.
    std::vector<int> tws = {tma::TWDEF};
    if (variant == 1) {
        auto area = [&](int tw) {
            return cdiv(g.nx - 1, tw) * tw * cdiv(g.ny - 2, tma::tile_h(tw)) * tma::tile_h(tw);
        };
        const long long amin = std::min(area(128), std::min(area(64), area(32)));
        tws.clear();
        for (int tw : {128, 64, 32})
            if (area(tw) == amin) tws.push_back(tw);
        best.tw = tws[0];
    }
    // A persistent launch balances its work queue only with a few items per
    // block: on a grid that fills the GPU alone, longer chunks that leave
    // fewer are not candidates.  A grid too small for that (fewer than four
    // items per resident block at the default chunk) shares its launches
    // with other systems when it is batched or served; its candidates are
    // timed on about a quarter as many blocks as they have items and ranked
    // by block-time (time x blocks), the share of a full launch they take.
    const long long blocks = variant == 1 ? (long long)tma_grid(g, 8).x : 0;
    const bool shared = variant == 1 && tma_items(g, kcs[0], tws[0]) < 4 * blocks;
    std::vector<std::pair<int, int>> cand;  // (tile width, z-chunk)
    for (int tw : tws) {
        const long long floor_items =
            variant == 1 ? std::min<long long>(tma_items(g, kcs[0], tw), 4 * blocks) : 0;
        for (int kc : kcs) {
            if (kc != kcs[0] && kc > g.nz - 2) continue;
            if (variant == 1 && !shared && kc != kcs[0] && tma_items(g, kc, tw) < floor_items)
                continue;
            cand.push_back({tw, kc});
        }
    }
    auto cand_blocks = [&](const std::pair<int, int> &c) -> unsigned {
        if (!shared) return 0u;
        const long long b = cdiv(tma_items(g, std::max(c.second, 4), c.first), 4);
        return (unsigned)std::max(1ll, std::min(b, blocks));
    };
    // clocks and caches to steady state, then round-robin timings (drift
    // during tuning then affects every candidate alike); median per candidate
    for (int i = 0; i < 12; ++i) tune_iter(sys, precision, variant, kcs[0], tws[0], i, s);
    const int rounds = 3;
    std::vector<std::vector<float>> t(cand.size());
    for (int r = 0; r < rounds; ++r)
        for (size_t c = 0; c < cand.size(); ++c) {
            float ms = 0.f;
            const unsigned nb = cand_blocks(cand[c]);
            if ((rc = time_candidate(sys, precision, variant, cand[c].second, cand[c].first, s,
                                     &ms, nb)) != PB_OK)
                return rc;
            t[c].push_back(shared ? ms * (float)nb : ms);
        }
    if (variant == 1) {
        // The timing runs never stop and leave arbitrary values (NaN after a
        // breakdown) in the FP32 vectors, also at the points past a row's
        // last tile that a wider candidate wrote and a narrower tile never
        // rewrites (the boundary column among them): clear them all.
        const size_t b32 = sizeof(float) * (size_t)g.Np;
        for (float *v : {sys->z32, sys->pa32, sys->pb32, sys->d32})
            PB_CUDA_TRY(cudaMemsetAsync(v, 0, b32, s));
    }
    float best_ms = 1e30f;
    for (size_t c = 0; c < cand.size(); ++c) {
        std::sort(t[c].begin(), t[c].end());
        const float ms = t[c][rounds / 2];
        // a candidate must beat the incumbent by 3% (timing noise would
        // otherwise make the choice, and the dot-product partition, vary)
        if (ms < 0.97f * best_ms) {
            best_ms = ms;
            best.tw = cand[c].first;
            best.kc = cand[c].second;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best;
    }
    *out = best;
    return PB_OK;
}

}  // namespace

pb_status set_tuning(pb_system *sys, int precision, int variant, int kc) {
    // kc = z-chunk + 10000 * tile width (0: the default width)
    const int tw = kc / 10000 ? kc / 10000 : tma::TWDEF;
    kc %= 10000;
    if (kc < 1 || variant < 0 || variant > 1 || !tma::tile_ok(tw) ||
        (variant == 1 && precision != PB_MIXED)) {
        set_error("bad tuning (variant %d, z-chunk %d, tile width %d)", variant, kc, tw);
        return PB_ERR_ARG;
    }
    const PadGeo &g = sys->pad;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    Tuning t;
    t.variant = variant;
    t.kc = kc;
    t.tw = tw;
    g_tune[std::make_tuple(precision, g.nx, g.ny, g.nz)] = t;
    return PB_OK;
}

pb_status set_wait_limit(long long polls) {
    const long long v = polls < 0 ? tma::TMA_WAIT_LIMIT : polls;
    PB_CUDA_TRY(cudaDeviceSynchronize());
    PB_CUDA_TRY(cudaMemcpyToSymbol(tma::g_slot_wait_limit, &v, sizeof(v)));
    PB_CUDA_TRY(cudaDeviceSynchronize());
    return PB_OK;
}

// work counters of the TMA stencil kernels ([0] next item, [1] finished
// blocks); zero between launches because each launch's last block resets them
pb_status ensure_queue(pb_system *sys, cudaStream_t s) {
    if (sys->queue) return PB_OK;
    sys->queue = (unsigned int *)dalloc(4 * sizeof(unsigned int), s);
    if (!sys->queue) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(sys->queue, 0, 4 * sizeof(unsigned int), s));
    return PB_OK;
}

pb_status ensure_solver_ws(pb_system *sys, int precision, cudaStream_t s) {
    const PadGeo &p = sys->pad;
    pb_status rc0 = PB_OK;
    if (!sys->st) {
        sys->st = (CgState *)dalloc(sizeof(CgState), s);
        if (!sys->st) return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(sys->st, 0, sizeof(CgState), s));
        PB_CUDA_TRY(cudaMallocHost((void **)&sys->h_st, 4 * sizeof(CgState)));
        dim3 g32 = stencil_grid<float>(p, 4), g64 = stencil_grid<double>(p, 4);
        long long nb = std::max<long long>((long long)g32.x * g32.y * g32.z,
                                           (long long)g64.x * g64.y * g64.z);
        nb = std::max<long long>(nb, cdiv(p.N, 256));
        sys->npartials = (int)(2 * nb + 64);
        sys->partials = (double *)dalloc(sizeof(double) * sys->npartials, s);
        if (!sys->partials) return PB_ERR_OOM;
        if ((rc0 = ensure_queue(sys, s)) != PB_OK) return rc0;
    }
    size_t bytes32 = sizeof(float) * (size_t)p.Np, bytes64 = sizeof(double) * (size_t)p.Np;
    if (precision == PB_MIXED && !sys->z32) {
        sys->z32 = (float *)dalloc(bytes32, s);
        sys->pa32 = (float *)dalloc(bytes32, s);
        sys->pb32 = (float *)dalloc(bytes32, s);
        sys->d32 = (float *)dalloc(bytes32, s);
        if (!sys->z32 || !sys->pa32 || !sys->pb32 || !sys->d32) return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(sys->z32, 0, bytes32, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->pa32, 0, bytes32, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->pb32, 0, bytes32, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->d32, 0, bytes32, s));
    }
    if (precision == PB_FP64 && !sys->z64) {
        sys->z64 = (double *)dalloc(bytes64, s);
        sys->pa64 = (double *)dalloc(bytes64, s);
        sys->pb64 = (double *)dalloc(bytes64, s);
        sys->x64 = (double *)dalloc(bytes64, s);
        if (!sys->z64 || !sys->pa64 || !sys->pb64 || !sys->x64) return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(sys->z64, 0, bytes64, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->pa64, 0, bytes64, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->pb64, 0, bytes64, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->x64, 0, bytes64, s));
    }
    if (precision == PB_FP64 && !sys->r64 && !sys->g->is_oct) {
        // the plain solver keeps r and q, and a padded copy of the operator
        sys->r64 = (double *)dalloc(bytes64, s);
        sys->q64 = (double *)dalloc(bytes64, s);
        for (int a = 0; a < 5; ++a) sys->op64[a] = (double *)dalloc(bytes64, s);
        if (!sys->r64 || !sys->q64 || !sys->op64[0] || !sys->op64[1] || !sys->op64[2] ||
            !sys->op64[3] || !sys->op64[4])
            return PB_ERR_OOM;
        PB_CUDA_TRY(cudaMemsetAsync(sys->r64, 0, bytes64, s));
        PB_CUDA_TRY(cudaMemsetAsync(sys->q64, 0, bytes64, s));
        k_cg64_operator<<<cdiv(p.Np, 256), 256, 0, s>>>(sys->W[0], sys->W[1], sys->W[2], sys->diag,
                                                         sys->g->geo, p, sys->op64[0], sys->op64[1],
                                                         sys->op64[2], sys->op64[3], sys->op64[4]);
        PB_LAUNCH_CHECK();
    }
    return PB_OK;
}

pb_status solve(pb_system *sys, const pb_solve_opts *o, cudaStream_t s, pb_solve_stats *stats) {
    double t_start = now_s();
    double deadline = o->time_budget_s > 0.0 ? t_start + o->time_budget_s : 0.0;
    const GridGeo &g = sys->g->geo;
    const PadGeo &p = sys->pad;
    pb_status rc = ensure_solver_ws(sys, o->precision, s);
    if (rc != PB_OK) return rc;
    if (o->precision == PB_MIXED && (rc = build_tma_state(sys)) != PB_OK) return rc;
    Tuning tune;
    if ((rc = autotune(sys, o->precision, s, &tune)) != PB_OK) return rc;
    int max_iter = o->max_iter > 0 ? o->max_iter : 100000;
    int max_outer = o->max_outer > 0 ? o->max_outer : 30;
    double rtol = o->rtol > 0.0 ? o->rtol : 1e-8;
    double inner_rtol = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-6;
    int chunk = 16;

    // phi = boundary values, interior 0 (zero initial guess)
    PB_CUDA_TRY(cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * g.N, cudaMemcpyDeviceToDevice, s));
    int iters = 0, outer = 0;
    int status = PB_OK;
    double fn2 = 0.0, res2 = 0.0;
    if (o->precision == PB_MIXED) {
        if ((rc = residual(sys, true, s)) != PB_OK) return rc;
        if ((rc = sync_state(sys, s)) != PB_OK) return rc;
        fn2 = sys->h_st->res64;
        res2 = fn2;
        outer = 1;
        CoefC32 cp = make_c32(sys);
        int stagnant = 0;
        while (fn2 > 0.0 && res2 > rtol * rtol * fn2) {
            if (outer > max_outer || iters >= max_iter) {
                status = PB_ERR_NOCONV;
                break;
            }
            double rel = sqrt(res2 / fn2);
            double itol = std::max(inner_rtol, 0.5 * rtol / rel);
            if (itol > 0.5) itol = 0.5;
            double rz = sys->h_st->rz64;
            if ((rc = init_state(sys, rz, res2, itol * itol * res2, max_iter - iters, s)) != PB_OK)
                return rc;
            size_t bytes32 = sizeof(float) * (size_t)p.Np;
            PB_CUDA_TRY(cudaMemsetAsync(sys->d32, 0, bytes32, s));
            PB_CUDA_TRY(cudaMemsetAsync(sys->pa32, 0, bytes32, s));
            int it = 0;
            rc = run_pcg<float, CoefC32>(sys, cp, sys->z32, sys->pa32, sys->pb32, sys->d32, tune.kc,
                                         tune.variant, tune.tw, chunk, deadline, s, &it);
            if (rc == PB_OK && sys->h_st[0].status == 3) {
                // the correction of an aborted inner solve is incomplete: it
                // is not promoted, phi keeps the last refined iterate
                set_error("a device-side wait reached its limit in the FP32 PCG kernels");
                status = PB_ERR_TIMEOUT;
                break;
            }
            if (rc == PB_ERR_TIMEOUT) {
                status = PB_ERR_TIMEOUT;
            } else if (rc != PB_OK) {
                return rc;
            }
            if (rc == PB_OK) iters += it;
            k_promote<float><<<cdiv(g.N, 256), 256, 0, s>>>(sys->phi, sys->d32, g, p);
            PB_LAUNCH_CHECK();
            if ((rc = residual(sys, true, s)) != PB_OK) return rc;
            if ((rc = sync_state(sys, s)) != PB_OK) return rc;
            double prev = res2;
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
        // plain FP64 PCG on the whole system, restarted from the true
        // residual if the recursive one drifted
        CoefS64 cp = make_s64(sys);
        size_t bytes64 = sizeof(double) * (size_t)p.Np;
        PB_CUDA_TRY(cudaMemsetAsync(sys->x64, 0, bytes64, s));
        if ((rc = residual(sys, false, s)) != PB_OK) return rc;
        if ((rc = sync_state(sys, s)) != PB_OK) return rc;
        fn2 = sys->h_st->res64;
        res2 = fn2;
        outer = 1;
        while (fn2 > 0.0 && res2 > rtol * rtol * fn2) {
            if (outer > max_outer || iters >= max_iter) {
                status = PB_ERR_NOCONV;
                break;
            }
            double rz = sys->h_st->rz64;
            if ((rc = init_state(sys, rz, res2, rtol * rtol * fn2 * 0.25, max_iter - iters, s)) != PB_OK)
                return rc;
            PB_CUDA_TRY(cudaMemsetAsync(sys->pa64, 0, bytes64, s));
            int it = 0;
            rc = run_pcg<double, CoefS64>(sys, cp, sys->z64, sys->pa64, sys->pb64, sys->x64, tune.kc,
                                          0, tma::TWDEF, chunk, deadline, s, &it);
            if (rc == PB_ERR_TIMEOUT) status = PB_ERR_TIMEOUT;
            else if (rc != PB_OK) return rc;
            if (rc == PB_OK) iters += it;
            PB_CUDA_TRY(cudaMemcpyAsync(sys->phi, sys->bc, sizeof(double) * g.N,
                                        cudaMemcpyDeviceToDevice, s));
            k_promote<double><<<cdiv(g.N, 256), 256, 0, s>>>(sys->phi, sys->x64, g, p);
            PB_LAUNCH_CHECK();
            if ((rc = residual(sys, false, s)) != PB_OK) return rc;
            if ((rc = sync_state(sys, s)) != PB_OK) return rc;
            res2 = sys->h_st->res64;
            ++outer;
            if (status == PB_ERR_TIMEOUT) break;
        }
    }
    sys->fnorm2 = fn2;
    sys->solved = 1;
    if (stats) {
        stats->status = status;
        stats->iters_inner = iters;
        stats->iters_outer = outer;
        stats->kc = tune.kc + 1000 * tune.variant + (tune.variant == 1 ? 10000 * tune.tw : 0);
        stats->true_rel_res = fn2 > 0.0 ? sqrt(res2 / fn2) : 0.0;
        stats->seconds = now_s() - t_start;
        stats->dof = (long long)(g.nx - 2) * (g.ny - 2) * (g.nz - 2);
        // FP32: P reads z,p_old writes p; U reads p,x,z writes x,z (+2 code bytes);
        // FP64 plain: same vectors plus three weight arrays streamed twice.
        long long per = o->precision == PB_MIXED ? (8 * 4 + 2) : (8 * 8 + 6 * 8 + 2);
        stats->model_bytes = (long long)iters * stats->dof * per + (long long)outer * g.N * 64;
    }
    return (pb_status)status;
}

void free_tma_state(pb_system *sys) {
    TmaState *t = (TmaState *)sys->tma;
    if (!t) return;
    dfree(t->dev, sys->stream);
    dfree(t->partials, sys->stream);
    dfree(t->cnt, sys->stream);
    delete t;
    sys->tma = nullptr;
}

pb_status profile_kernels(pb_system *sys, int precision, int which, int reps, cudaStream_t s) {
    if (precision == PB_MIXED && !sys->z32) {
        set_error("no mixed-precision solver state");
        return PB_ERR_STATE;
    }
    if (precision == PB_FP64 && !sys->z64) {
        set_error("no FP64 solver state");
        return PB_ERR_STATE;
    }
    pb_status rc = PB_OK;
    if (precision == PB_MIXED && (rc = build_tma_state(sys)) != PB_OK) return rc;
    Tuning tune;
    if ((rc = autotune(sys, precision, s, &tune)) != PB_OK) return rc;
    if ((rc = init_state(sys, 1.0, 1.0, -1.0, 1 << 30, s, 1)) != PB_OK) return rc;
    const int KC = tune.kc;
    for (int r = 0; r < reps; ++r) {
        const int cur = r & 1;
        if (precision == PB_MIXED && tune.variant == 1) {
            TmaState *t = (TmaState *)sys->tma;
            if ((rc = tma_use_kc(sys, KC, tune.tw, s)) != PB_OK) return rc;
            dim3 grid = tma_grid(sys->pad, KC);
            if (which == 0 || which == 2) {
                tma_launch<MODE_P>(t->dev, 1, t->host.nitems, sys->queue, grid, s, &t->host, true);
                PB_LAUNCH_CHECK();
            }
            if (which == 1 || which == 2) {
                tma_launch<MODE_U>(t->dev, 1, t->host.nitems, sys->queue, grid, s, &t->host, true);
                PB_LAUNCH_CHECK();
            }
        } else if (precision == PB_MIXED) {
            CoefC32 cp = make_c32(sys);
            dim3 grid = stencil_grid<float>(sys->pad, KC);
            KArgs<float> a{};
            a.code = sys->code;
            a.st = sys->st;
            a.partials = sys->partials;
            a.pg = sys->pad;
            a.KC = KC;
            float *pbuf[2] = {sys->pa32, sys->pb32};
            if (which == 0 || which == 2) {
                a.in = sys->z32;
                a.in2 = pbuf[cur];
                a.out = pbuf[cur ^ 1];
                k_stencil<float, CoefC32, MODE_P, TYC, MinB<float>::v><<<grid, 32 * TYC, 0, s>>>(a, cp);
                PB_LAUNCH_CHECK();
            }
            if (which == 1 || which == 2) {
                a.in = pbuf[cur ^ 1];
                a.in2 = nullptr;
                a.out = nullptr;
                a.xv = sys->d32;
                a.zv = sys->z32;
                k_stencil<float, CoefC32, MODE_U, TYC, MinB<float>::v><<<grid, 32 * TYC, 0, s>>>(a, cp);
                PB_LAUNCH_CHECK();
            }
        } else {
            launch_iter_cg64(sys, cur, KC, s, which);
            note_launch(which == 2 ? 1 : 0);
            PB_LAUNCH_CHECK();
        }
    }
    // phi is untouched: only the solver workspace (z, p, x increment) changed
    return PB_OK;
}

pb_status apply_op(pb_system *sys, int precision, const void *x, void *y, cudaStream_t s) {
    const GridGeo &g = sys->g->geo;
    const PadGeo &p = sys->pad;
    int KC = default_kc(p, precision);
    size_t esz = precision == PB_MIXED ? 4 : 8;
    void *xp = dalloc(esz * (size_t)p.Np, s), *yp = dalloc(esz * (size_t)p.Np, s);
    if (!xp || !yp) return PB_ERR_OOM;
    PB_CUDA_TRY(cudaMemsetAsync(xp, 0, esz * (size_t)p.Np, s));
    PB_CUDA_TRY(cudaMemsetAsync(yp, 0, esz * (size_t)p.Np, s));
    unsigned blocks = cdiv(g.N, 256);
    if (precision == PB_MIXED) {
        k_canon_to_pad<float><<<blocks, 256, 0, s>>>((const float *)x, (float *)xp, g, p);
        if (ensure_queue(sys, s) != PB_OK) return PB_ERR_OOM;
        // a one-entry table of its own (the solver's entry may be in use)
        tma::SysEntry *e = new (std::nothrow) tma::SysEntry();
        if (!e) return PB_ERR_OOM;
        pb_status rc =
            tma_maps(sys, MODE_A, (const float *)xp, nullptr, nullptr, nullptr, &e->A, tma::TWDEF);
        if (rc == PB_OK) rc = tma_prepare<MODE_A>();
        if (rc != PB_OK) {
            delete e;
            return rc;
        }
        e->pg = p;
        e->cp = make_c32(sys);
        e->y = (float *)yp;
        tma_entry_geometry(*e, p, 8, tma::TWDEF);
        tma::SysEntry *de = (tma::SysEntry *)dalloc(sizeof(tma::SysEntry), s);
        if (!de) {
            delete e;
            return PB_ERR_OOM;
        }
        cudaError_t ce = cudaMemcpyAsync(de, e, sizeof(tma::SysEntry), cudaMemcpyHostToDevice, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        const int nitems = e->nitems;
        if (ce != cudaSuccess) {
            delete e;
            set_error("apply table upload: %s", cudaGetErrorString(ce));
            return PB_ERR_CUDA;
        }
        tma_launch<MODE_A>(de, 1, nitems, sys->queue, tma_grid(p, 8), s, e);
        delete e;
        PB_LAUNCH_CHECK();
        dfree(de, s);
        k_pad_to_canon<float><<<blocks, 256, 0, s>>>((const float *)yp, (float *)y, g, p);
    } else {
        k_canon_to_pad<double><<<blocks, 256, 0, s>>>((const double *)x, (double *)xp, g, p);
        KArgs<double> a{};
        a.in = (const double *)xp;
        a.out = (double *)yp;
        a.code = sys->code;
        a.pg = p;
        a.KC = KC;
        k_stencil<double, CoefS64, MODE_A, TYC, MinB<double>::v><<<stencil_grid<double>(p, KC), 32 * TYC, 0, s>>>(
            a, make_s64(sys));
        k_pad_to_canon<double><<<blocks, 256, 0, s>>>((const double *)yp, (double *)y, g, p);
    }
    note_launch(2);
    PB_LAUNCH_CHECK();
    dfree(xp, s);
    dfree(yp, s);
    return PB_OK;
}

}  // namespace pbg

namespace pbg {

#include "engine.cuh"
#include "split.cuh"

// Batched mixed-precision solve through the continuous-batching engine: every
// system takes a slot of one launch table, whose PCG iterations run as
// replays of one captured graph, and each system's FP64 refinement steps are
// decided on the device (k_ir_step) as soon as its own inner solve ends, so
// no system waits for another's.  The host only watches the pinned state
// mirror.  A system's arithmetic is the same as in pb_solve with the same
// tuning, so its result does not depend on the batch (uniform and octree
// systems alike).
pb_status solve_batch(pb_system *const *systems, int n, const pb_solve_opts *o, cudaStream_t s,
                      pb_solve_stats *stats) {
    const double t_start = now_s();
    const double deadline = o->time_budget_s > 0.0 ? t_start + o->time_budget_s : 0.0;
    pb_engine *eh = nullptr;
    pb_status rc = engine_create(systems[0]->g->device, n, o, &eh);
    if (rc != PB_OK) return rc;
    std::map<long long, int> index;
    std::vector<int> got(n, 0);
    for (int i = 0; i < n && rc == PB_OK; ++i) {
        long long t = 0;
        rc = engine_submit(eh, systems[i], s, &t);
        if (rc == PB_OK) index[t] = i;
    }
    int left = rc == PB_OK ? n : 0;
    bool timed_out = false;
    std::vector<pb_engine_result> out(std::max(n, 1));
    while (left > 0) {
        double wait = 0.05;
        if (deadline > 0.0) {
            const double rem = deadline - now_s();
            if (rem <= 0.0) {
                timed_out = true;
                break;
            }
            wait = std::min(wait, rem);
        }
        int k = 0;
        pb_status r = engine_wait(eh, wait, out.data(), n, &k);
        if (r != PB_OK) {
            rc = r;
            break;
        }
        for (int q = 0; q < k; ++q) {
            auto it = index.find(out[q].ticket);
            if (it == index.end()) continue;
            const int i = it->second;
            stats[i] = out[q].stats;
            got[i] = 1;
            --left;
        }
    }
    // stops the pump; systems still in the table get their own state back
    engine_destroy(eh);
    pb_status worst = PB_OK;
    for (int i = 0; i < n; ++i) {
        if (!got[i]) {
            stats[i] = pb_solve_stats{};
            stats[i].status = rc != PB_OK ? rc : PB_ERR_TIMEOUT;
            stats[i].seconds = now_s() - t_start;
        }
        if (stats[i].status != PB_OK) worst = (pb_status)stats[i].status;
    }
    if (rc != PB_OK) return rc;
    if (timed_out && worst == PB_OK) worst = PB_ERR_TIMEOUT;
    return worst;
}


}  // namespace pbg
