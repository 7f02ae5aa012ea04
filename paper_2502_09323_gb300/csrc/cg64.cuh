// Plain FP64 Jacobi-PCG kernels (included by solve.cu inside its anonymous
// namespace; needs CgState, PadGeo and last_block_total from there).
//
// The textbook preconditioned CG (Sec. 4) with the Jacobi preconditioner,
// every vector and every operation in FP64, one solve at a time:
//   kernel D:  p = z + beta p_old ;  q = A p ;  sigma = p.q       -> alpha = rho / sigma
//   kernel U:  x += alpha p ;  r -= alpha q ;  z = D^-1 r ;
//              rho' = r.z ;  rr = r.r                            -> beta = rho' / rho
// GB300's FP64 pipe (about 1/64 of the FP32 rate) binds before HBM does, so
// the schedule keeps FP64 operations per unknown and iteration low: the
// operator is applied once per iteration (q is stored), and the diagonal
// and its inverse are stored, so there is no division and no diagonal
// rebuilt from the six weights.  Per unknown: D does 11 FP64 operations (p
// on the own row and on the two rows next to it, 1 multiply and 6
// multiply-adds for A p, 1 for sigma) and U does 5; the traffic is 16 FP64
// words (128 B): D reads z, p_old, three weights and the diagonal and writes
// p and q, U reads x, r, p, q and the inverse diagonal and writes x, r and z.
//
// Layout: every array is padded (rows of sx elements, 16-byte aligned), zero
// off the interior (z, r, p, q, and the diagonal and its inverse), so that
// boundary neighbours contribute nothing to A p (their values are lifted into
// f) and U needs no interior test.  Each reduction is summed per thread and
// block in FP64 and across blocks by the last block in a fixed order: the
// results are identical run to run.
#pragma once

namespace cg64 {

constexpr int WARPS = 8;            // rows per block
constexpr int NT = 32 * WARPS;
constexpr int TXP = 64;             // points per row and block: two per lane
constexpr int UNT = 256;            // threads of the update kernel

struct DirArgs {
    const double *z, *pold;
    double *p, *q;
    const double *w0, *w1, *w2;     // +x, +y, +z edge weight of each node
    const double *dg;               // diagonal
    CgState *st;
    double *partials;
    PadGeo g;
    int KC;                         // planes per block
};

struct UpdArgs {
    double *x, *r, *z;
    const double *p, *q, *dinv;
    CgState *st;
    double *partials;
    long long first, count;         // slots [first, first + count), count even
};

__device__ __forceinline__ double2 ld2(const double *a, int i) {
    return *reinterpret_cast<const double2 *>(a + i);
}

}  // namespace cg64

// Direction kernel.  Each warp owns one row j (64 points, two per lane) of a
// 64 x 8 tile and marches over KC planes, keeping its row of p at planes
// k-1, k, k+1 in registers; rows j-1 and j+1 of plane k are formed from z and
// p_old read through L1/L2 (their own warps streamed them from HBM), x
// neighbours come from shuffles and one scalar load at each tile edge, and
// the -z weight is the +z weight of the previous plane.  Loads of plane k+1
// (neighbour rows) and k+2 (own row) are issued before plane k is computed.
__global__ void __launch_bounds__(cg64::NT, 2) k_cg64_dir(cg64::DirArgs A) {
    using namespace cg64;
    __shared__ double sred[NT / 32];
    if (A.st->done) return;  // changes only at the end of a launch
    const double beta = A.st->beta;
    const PadGeo g = A.g;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * TXP;
    const int ib = i0 + 2 * lane;
    const int j = 1 + blockIdx.y * WARPS + w;
    const int k0 = 1 + blockIdx.z * A.KC;
    const int k1 = min(k0 + A.KC, g.nz - 1);
    const bool grp = j <= g.ny - 2 && ib < g.sx;
    const bool hl = j <= g.ny - 2 && lane == 0 && i0 > 0;
    const bool hr = j <= g.ny - 2 && lane == 31 && i0 + TXP < g.sx;
    const int sx = g.sx, sxy = (int)g.sxy;
    // interior points of this lane
    const bool in0 = grp && ib >= 1 && ib <= g.nx - 2;
    const bool in1 = grp && ib + 1 >= 1 && ib + 1 <= g.nx - 2;

    auto pform = [&](double2 zz, double2 po) {
        return make_double2(fma(beta, po.x, zz.x), fma(beta, po.y, zz.y));
    };
    const double2 zero2 = make_double2(0.0, 0.0);
    double2 pm = zero2, pc = zero2, pn = zero2, ym = zero2, yp = zero2, w2m = zero2;
    double lc = 0.0, rc = 0.0;
    if (grp) {
        const int b0 = (k0 - 1) * sxy + j * sx + ib;
        pm = pform(ld2(A.z, b0), ld2(A.pold, b0));
        pc = pform(ld2(A.z, b0 + sxy), ld2(A.pold, b0 + sxy));
        pn = pform(ld2(A.z, b0 + 2 * sxy), ld2(A.pold, b0 + 2 * sxy));
        ym = pform(ld2(A.z, b0 + sxy - sx), ld2(A.pold, b0 + sxy - sx));
        yp = pform(ld2(A.z, b0 + sxy + sx), ld2(A.pold, b0 + sxy + sx));
        w2m = ld2(A.w2, b0);
    }
    if (hl) {
        const int q0 = k0 * sxy + j * sx + i0 - 1;
        lc = fma(beta, A.pold[q0], A.z[q0]);
    }
    if (hr) {
        const int q0 = k0 * sxy + j * sx + i0 + TXP;
        rc = fma(beta, A.pold[q0], A.z[q0]);
    }
    double acc = 0.0;
    for (int k = k0; k < k1; ++k) {
        const int base = k * sxy + j * sx;
        const bool more = k + 1 < k1;
        // ---- loads: the next planes' vectors and this plane's coefficients
        double2 zn2 = zero2, on2 = zero2, zym = zero2, oym = zero2, zyp = zero2, oyp = zero2;
        double lz = 0.0, lo = 0.0, rz = 0.0, ro = 0.0, wl = 0.0;
        double2 w0c = zero2, w1c = zero2, w1m = zero2, w2c = zero2, dgc = zero2;
        if (grp) {
            const int q = base + ib;
            if (more) {
                zn2 = ld2(A.z, q + 2 * sxy);
                on2 = ld2(A.pold, q + 2 * sxy);
                zym = ld2(A.z, q + sxy - sx);
                oym = ld2(A.pold, q + sxy - sx);
                zyp = ld2(A.z, q + sxy + sx);
                oyp = ld2(A.pold, q + sxy + sx);
            }
            w0c = ld2(A.w0, q);
            w1c = ld2(A.w1, q);
            w1m = ld2(A.w1, q - sx);
            w2c = ld2(A.w2, q);
            dgc = ld2(A.dg, q);
        }
        if (hl) {
            wl = A.w0[base + i0 - 1];
            if (more) {
                lz = A.z[base + sxy + i0 - 1];
                lo = A.pold[base + sxy + i0 - 1];
            }
        }
        if (hr && more) {
            rz = A.z[base + sxy + i0 + TXP];
            ro = A.pold[base + sxy + i0 + TXP];
        }
        // ---- q = A p on plane k
        double left = __shfl_up_sync(0xffffffffu, pc.y, 1);
        double right = __shfl_down_sync(0xffffffffu, pc.x, 1);
        double wxl = __shfl_up_sync(0xffffffffu, w0c.y, 1);
        if (lane == 0) {
            left = lc;
            wxl = wl;
        }
        if (lane == 31) right = rc;
        double q0 = dgc.x * pc.x;
        q0 = fma(-wxl, left, q0);
        q0 = fma(-w0c.x, pc.y, q0);
        q0 = fma(-w1m.x, ym.x, q0);
        q0 = fma(-w1c.x, yp.x, q0);
        q0 = fma(-w2m.x, pm.x, q0);
        q0 = fma(-w2c.x, pn.x, q0);
        double q1 = dgc.y * pc.y;
        q1 = fma(-w0c.x, pc.x, q1);
        q1 = fma(-w0c.y, right, q1);
        q1 = fma(-w1m.y, ym.y, q1);
        q1 = fma(-w1c.y, yp.y, q1);
        q1 = fma(-w2m.y, pm.y, q1);
        q1 = fma(-w2c.y, pn.y, q1);
        q0 = in0 ? q0 : 0.0;
        q1 = in1 ? q1 : 0.0;
        acc = fma(pc.x, q0, acc);
        acc = fma(pc.y, q1, acc);
        if (grp) {
            *reinterpret_cast<double2 *>(A.p + base + ib) = pc;
            *reinterpret_cast<double2 *>(A.q + base + ib) = make_double2(q0, q1);
        }
        // ---- rotate
        pm = pc;
        pc = pn;
        w2m = w2c;
        if (more) {
            pn = pform(zn2, on2);
            ym = pform(zym, oym);
            yp = pform(zyp, oyp);
            lc = hl ? fma(beta, lo, lz) : 0.0;
            rc = hr ? fma(beta, ro, rz) : 0.0;
        }
    }
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    double t0, t1;
    if (last_block_total<NT, false>(A.st, A.partials, nb, acc, 0.0, sred, t0, t1)) {
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
}

// Update kernel: streams the interior planes (boundary rows and padding hold
// zeros, so they need no test), two slots per thread and loop step.
__global__ void __launch_bounds__(cg64::UNT, 4) k_cg64_upd(cg64::UpdArgs A) {
    using namespace cg64;
    __shared__ double sred[UNT / 32];
    if (A.st->done) return;
    const double alpha = A.st->alpha;
    double rho = 0.0, rr = 0.0;
    const long long n2 = A.count >> 1;
    const long long stride = (long long)gridDim.x * UNT;
    for (long long t = blockIdx.x * (long long)UNT + threadIdx.x; t < n2; t += stride) {
        const long long e = A.first + 2 * t;
        double2 x = *reinterpret_cast<const double2 *>(A.x + e);
        double2 r = *reinterpret_cast<const double2 *>(A.r + e);
        const double2 p = *reinterpret_cast<const double2 *>(A.p + e);
        const double2 q = *reinterpret_cast<const double2 *>(A.q + e);
        const double2 di = *reinterpret_cast<const double2 *>(A.dinv + e);
        x.x = fma(alpha, p.x, x.x);
        x.y = fma(alpha, p.y, x.y);
        r.x = fma(-alpha, q.x, r.x);
        r.y = fma(-alpha, q.y, r.y);
        const double2 z = make_double2(di.x * r.x, di.y * r.y);
        rho = fma(r.x, z.x, rho);
        rho = fma(r.y, z.y, rho);
        rr = fma(r.x, r.x, rr);
        rr = fma(r.y, r.y, rr);
        *reinterpret_cast<double2 *>(A.x + e) = x;
        *reinterpret_cast<double2 *>(A.r + e) = r;
        *reinterpret_cast<double2 *>(A.z + e) = z;
    }
    const int nb = gridDim.x;
    double t0, t1;
    if (last_block_total<UNT, true>(A.st, A.partials, nb, rho, rr, sred, t0, t1)) {
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

// Padded FP64 operator of the plain solver: the three weights, the diagonal
// and its inverse at interior nodes, zero elsewhere (padding included).
__global__ void k_cg64_operator(const double *__restrict__ W0, const double *__restrict__ W1,
                                const double *__restrict__ W2, const double *__restrict__ diag,
                                GridGeo g, PadGeo pg, double *w0, double *w1, double *w2, double *dg,
                                double *dinv) {
    const long long a = blockIdx.x * 256ll + threadIdx.x;
    if (a >= pg.Np) return;
    const long long i = a % pg.sx, j = (a / pg.sx) % pg.ny, k = a / pg.sxy;
    const bool interior = i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
    const long long c = (k * g.ny + j) * g.nx + i;
    w0[a] = interior ? W0[c] : 0.0;
    w1[a] = interior ? W1[c] : 0.0;
    w2[a] = interior ? W2[c] : 0.0;
    dg[a] = interior ? diag[c] : 0.0;
    dinv[a] = interior ? 1.0 / diag[c] : 0.0;
}
