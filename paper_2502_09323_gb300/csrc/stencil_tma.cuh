// FP32 PCG stencil kernels with TMA staging (included by solve.cu).
//
// A block covers a tile of 128 x nodes by 8 rows and marches along z over KC
// planes.  One producer warp (lane 0) issues, for every plane, tensor-map
// (cp.async.bulk.tensor) loads of
//   * the streamed vector on a 136 x 10 box (4 columns of x halo on each side
//     and one halo row above and below; out-of-range elements are zero),
//   * for the update kernel, the x and z rows of the tile (128 x 8),
//   * the code bytes on a 160 x 10 box,
// into a ring of NSLOT shared-memory slots, each guarded by a "full" mbarrier
// (transaction bytes) and an "empty" mbarrier (one arrival per consumer warp).
// The 8 consumer warps compute one row each; a warp holds at most two slots
// (planes k and k+1) and keeps its own row of planes k-1, k in registers, so
// the producer runs up to NSLOT-2 planes ahead of the slowest warp.  No
// consumer ever waits on another consumer.
//
// Every wait is bounded: after TMA_WAIT_LIMIT polls a wait gives up, the
// block records status 3 in the solver state, stops, waits (bounded) for its
// own copies still in flight, and returns.
// Included inside solve.cu's anonymous namespace (needs KArgs, CoefC32,
// CgState and last_block_total from there).
#pragma once

namespace tma {

constexpr int ROWS = 8;              // consumer warps = tile rows
constexpr int NSLOT = 4;             // ring depth
constexpr int BOXW = 136;            // streamed box width (floats), x from i0-4
constexpr int OWNW = 128;            // own-row box width (floats), x from i0
constexpr int CODEW = 160;           // code box width (bytes), x from i0-16
constexpr int BOXH = ROWS + 2;       // rows j0-1 .. j0+ROWS
constexpr int NTHREADS = 32 * (ROWS + 1);
constexpr long long TMA_WAIT_LIMIT = 1ll << 20;

constexpr int align128(int b) { return (b + 127) & ~127; }
constexpr int BOX_BYTES = BOXW * BOXH * 4;    // 5440
constexpr int OWN_BYTES = OWNW * ROWS * 4;    // 4096
constexpr int CODE_BYTES = CODEW * BOXH;      // 1600

template <int MODE>
struct SlotLayout;
// direction kernel: z and p_old boxes + codes
template <>
struct SlotLayout<0> {
    static constexpr int a = 0, b = align128(BOX_BYTES), x = -1, z = -1,
                         code = 2 * align128(BOX_BYTES);
    static constexpr int stride = align128(code + CODE_BYTES);
    static constexpr unsigned tx = 2 * BOX_BYTES + CODE_BYTES;
};
// update kernel: p box, x and z rows, codes
template <>
struct SlotLayout<1> {
    static constexpr int a = 0, b = -1, x = align128(BOX_BYTES), z = x + OWN_BYTES,
                         code = z + OWN_BYTES;
    static constexpr int stride = align128(code + CODE_BYTES);
    static constexpr unsigned tx = BOX_BYTES + 2 * OWN_BYTES + CODE_BYTES;
};
// apply: x box + codes
template <>
struct SlotLayout<2> {
    static constexpr int a = 0, b = -1, x = -1, z = -1, code = align128(BOX_BYTES);
    static constexpr int stride = align128(code + CODE_BYTES);
    static constexpr unsigned tx = BOX_BYTES + CODE_BYTES;
};

template <int MODE>
constexpr int smem_bytes() {
    return NSLOT * SlotLayout<MODE>::stride + 2 * NSLOT * 8;
}

struct Maps {
    CUtensorMap a;      // streamed vector, 136 x 10 box (P: z, U: p, A: x)
    CUtensorMap b;      // P: p_old, 136 x 10 box
    CUtensorMap x;      // U: x, 128 x 8 box
    CUtensorMap z;      // U: z, 128 x 8 box
    CUtensorMap code;   // 160 x 10 box of code bytes
};

// ------------------------------------------------------------------- PTX --
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the limit was reached
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long n = 0; n < TMA_WAIT_LIMIT; ++n)
        if (mbar_try(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

}  // namespace tma

// MODE_P / MODE_U / MODE_A on the compressed FP32 operator.
template <int MODE>
__global__ void __launch_bounds__(tma::NTHREADS, 3)
k_stencil_tma(const __grid_constant__ tma::Maps maps, KArgs<float> A, CoefC32 cp) {
    using namespace tma;
    using L = SlotLayout<MODE>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ double sred[NTHREADS / 32];
    __shared__ int s_abort;

    float alpha = 0.f, beta = 0.f;
    if (MODE != MODE_A) {
        if (A.st->done) return;
        if (MODE == MODE_P) beta = (float)A.st->beta;
        if (MODE == MODE_U) alpha = (float)A.st->alpha;
    }
    const PadGeo g = A.pg;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * OWNW;
    const int j0 = 1 + blockIdx.y * ROWS;
    const int k0 = 1 + blockIdx.z * A.KC;
    const int k1 = min(k0 + A.KC, g.nz - 1);
    const int nplanes = (k1 - k0) + 2;  // planes k0-1 .. k1
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NSLOT * L::stride);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSLOT);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, ROWS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();

    float acc0 = 0.f, acc1 = 0.f;
    if (w == ROWS) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            int last_use[NSLOT];
            for (int s = 0; s < NSLOT; ++s) last_use[s] = -1;
            for (int t = 0; t < nplanes; ++t) {
                const int s = t % NSLOT, u = t / NSLOT;
                if (u > 0 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1)) {
                    s_abort = 1;
                    break;
                }
                if (*(volatile int *)&s_abort) break;
                const uint32_t bar = full0 + 8 * s;
                const uint32_t slot = smem_u32(smem + s * L::stride);
                const int kp = k0 - 1 + t;
                mbar_expect_tx(bar, L::tx);
                tma_load3(slot + L::a, &maps.a, i0 - 4, j0 - 1, kp, bar);
                if (MODE == MODE_P) tma_load3(slot + L::b, &maps.b, i0 - 4, j0 - 1, kp, bar);
                if (MODE == MODE_U) {
                    tma_load3(slot + L::x, &maps.x, i0, j0, kp, bar);
                    tma_load3(slot + L::z, &maps.z, i0, j0, kp, bar);
                }
                tma_load3(slot + L::code, &maps.code, i0 - 16, j0 - 1, kp, bar);
                last_use[s] = u;
            }
            // drain: every armed slot's copies must land before the block exits
            for (int s = 0; s < NSLOT; ++s)
                if (last_use[s] >= 0) mbar_wait(full0 + 8 * s, last_use[s] & 1);
        }
    } else {
        // ------------------------------------------------------- consumers
        const int j = j0 + w;
        const int r = w + 1;  // this row inside the halo boxes
        const int ib = i0 + lane * 4;
        const bool active = j <= g.ny - 2;
        const bool grp_ok = active && ib < g.sx;
        const float dg_in = 6.f * cp.w_in, dg_out = 6.f * cp.w_out + cp.kap;
        const float dinv_in = 1.f / dg_in, dinv_out = 1.f / dg_out;

        auto slot_ptr = [&](int t) { return smem + (t % NSLOT) * L::stride; };
        auto wait_full = [&](int t) -> bool {
            if (!mbar_wait(full0 + 8 * (t % NSLOT), (t / NSLOT) & 1)) {
                s_abort = 1;
                return false;
            }
            return !*(volatile int *)&s_abort;
        };
        auto release = [&](int t) {
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * (t % NSLOT));
        };
        // streamed value (P: z + beta p_old) of box row rr at box column cc
        auto val4 = [&](const uint8_t *sl, int rr, float (&v)[4]) {
            const float *a = reinterpret_cast<const float *>(sl + L::a) + rr * BOXW + 4 + lane * 4;
            float4 t = *reinterpret_cast<const float4 *>(a);
            v[0] = t.x;
            v[1] = t.y;
            v[2] = t.z;
            v[3] = t.w;
            if (MODE == MODE_P) {
                const float *b = reinterpret_cast<const float *>(sl + L::b) + rr * BOXW + 4 + lane * 4;
                float4 u = *reinterpret_cast<const float4 *>(b);
                v[0] += beta * u.x;
                v[1] += beta * u.y;
                v[2] += beta * u.z;
                v[3] += beta * u.w;
            }
        };
        auto val1 = [&](const uint8_t *sl, int rr, int col) -> float {
            float v = reinterpret_cast<const float *>(sl + L::a)[rr * BOXW + col];
            if (MODE == MODE_P) v += beta * reinterpret_cast<const float *>(sl + L::b)[rr * BOXW + col];
            return v;
        };
        auto code4 = [&](const uint8_t *sl, int rr) -> uint32_t {
            return *reinterpret_cast<const uint32_t *>(sl + L::code + rr * CODEW + 16 + lane * 4);
        };

        float pm[4], pc[4], pn[4];
        uint32_t cm = 0, cc = 0, cn = 0;
        // +z weights of this row at plane k-1 (the -z weights of plane k).
        // A plane on the fast path has no listed +z edge, so its pure +z
        // weights are exact too; only the first plane of a chunk loads them.
        float wzc[4] = {0.f, 0.f, 0.f, 0.f};
        bool ok = wait_full(0);
        if (ok) {
            const uint8_t *s0 = slot_ptr(0);
            val4(s0, r, pm);
            cm = code4(s0, r);
            release(0);
            ok = wait_full(1);
        }
        if (ok) {
            const uint8_t *s1 = slot_ptr(1);
            val4(s1, r, pc);
            cc = code4(s1, r);
        }
        for (int t = 1; ok && t <= k1 - k0; ++t) {
            const int k = k0 + t - 1;
            if (!wait_full(t + 1)) break;
            const uint8_t *sc = slot_ptr(t), *sn = slot_ptr(t + 1);
            val4(sn, r, pn);
            cn = code4(sn, r);
            float ym[4], yp[4];
            val4(sc, r - 1, ym);
            val4(sc, r + 1, yp);
            const uint32_t cym = code4(sc, r - 1);
            float left = __shfl_up_sync(0xffffffffu, pc[3], 1);
            float right = __shfl_down_sync(0xffffffffu, pc[0], 1);
            if (lane == 0) left = val1(sc, r, 3);
            if (lane == 31) right = val1(sc, r, 4 + 32 * 4);
            const uint32_t lcode = sc[L::code + r * CODEW + 15 + lane * 4];
            float xv[4] = {0.f, 0.f, 0.f, 0.f}, zv[4] = {0.f, 0.f, 0.f, 0.f};
            if (MODE == MODE_U) {
                float4 a = *reinterpret_cast<const float4 *>(sc + L::x + (w * OWNW + lane * 4) * 4);
                float4 b = *reinterpret_cast<const float4 *>(sc + L::z + (w * OWNW + lane * 4) * 4);
                xv[0] = a.x;
                xv[1] = a.y;
                xv[2] = a.z;
                xv[3] = a.w;
                zv[0] = b.x;
                zv[1] = b.y;
                zv[2] = b.z;
                zv[3] = b.w;
            }
            const uint32_t cxl = (cc << 8) | lcode;
            const uint32_t special = (cc & 0x0E0E0E0Eu) | (cxl & 0x02020202u) |
                                     (cym & 0x04040404u) | (cm & 0x08080808u);
            const bool fast = !__any_sync(0xffffffffu, special != 0u);
            const int base = k * (int)g.sxy + j * g.sx;
            // per-point weights of the six faces
            float wxp[4], wxm[4], wyp[4], wym[4], wzp[4], wzm[4];
            if (fast) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float wp = cp.pure((uint8_t)(cc >> (8 * q)));
                    wxp[q] = wxm[q] = wyp[q] = wym[q] = wzp[q] = wzm[q] = wp;
                }
            } else {
                const bool wz_valid = t > 1;
                // issue every listed-weight load first, then use them
                const int pl = base + ib;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint8_t c0 = (uint8_t)(cc >> (8 * q));
                    const float wp = cp.pure(c0);
                    wxp[q] = (c0 & 2) ? __ldg(cp.wx + pl + q) : wp;
                    wyp[q] = (c0 & 4) ? __ldg(cp.wy + pl + q) : wp;
                    wzp[q] = (c0 & 8) ? __ldg(cp.wz + pl + q) : wp;
                    const uint8_t cy = (uint8_t)(cym >> (8 * q));
                    wym[q] = (cy & 4) ? __ldg(cp.wy + pl + q - g.sx) : wp;
                    const uint8_t cz = (uint8_t)(cm >> (8 * q));
                    wzm[q] = wz_valid ? wzc[q]
                                      : ((cz & 8) ? __ldg(cp.wz + pl + q - (int)g.sxy) : wp);
                }
                // -x weight of point q is the +x weight of point q-1
                float wl = __shfl_up_sync(0xffffffffu, wxp[3], 1);
                if (lane == 0) {
                    const uint8_t c0 = (uint8_t)cc;
                    wl = (lcode & 2) ? __ldg(cp.wx + pl - 1) : cp.pure(c0);
                }
                wxm[0] = wl;
                wxm[1] = wxp[0];
                wxm[2] = wxp[1];
                wxm[3] = wxp[2];
            }
            float y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = ib + q;
                const uint8_t c0 = (uint8_t)(cc >> (8 * q));
                const float x0 = pc[q];
                const float xl = q > 0 ? pc[q - 1] : left;
                const float xr = q < 3 ? pc[q + 1] : right;
                const float kp = cp.kappa(c0);
                float ap, dinv, dg;
                if (fast) {
                    const float wp = wxp[q];
                    const float sum = ((x0 - xl) + (x0 - xr)) + ((x0 - ym[q]) + (x0 - yp[q])) +
                                      ((x0 - pm[q]) + (x0 - pn[q]));
                    ap = wp * sum + kp * x0;
                    dinv = (c0 & 1) ? dinv_in : dinv_out;
                    dg = (c0 & 1) ? dg_in : dg_out;
                } else {
                    ap = kp * x0;
                    ap += wxm[q] * (x0 - xl);
                    ap += wxp[q] * (x0 - xr);
                    ap += wym[q] * (x0 - ym[q]);
                    ap += wyp[q] * (x0 - yp[q]);
                    ap += wzm[q] * (x0 - pm[q]);
                    ap += wzp[q] * (x0 - pn[q]);
                    dg = ((((((wxm[q] + wxp[q]) + wym[q]) + wyp[q]) + wzm[q]) + wzp[q]) + kp);
                    dinv = 1.f / dg;
                }
                const bool interior = grp_ok && i >= 1 && i <= g.nx - 2;
                y[q] = interior ? ap : 0.f;
                if (MODE == MODE_P) {
                    if (interior) acc0 += x0 * ap;
                } else if (MODE == MODE_U) {
                    if (interior) {
                        xv[q] = xv[q] + alpha * x0;
                        const float znew = zv[q] - alpha * ap * dinv;
                        zv[q] = znew;
                        const float rr = dg * znew;
                        acc0 += rr * znew;
                        acc1 += rr * rr;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) wzc[q] = wzp[q];
            release(t);
            if (grp_ok) {
                if (MODE == MODE_P)
                    *reinterpret_cast<float4 *>(A.out + base + ib) = make_float4(pc[0], pc[1], pc[2], pc[3]);
                if (MODE == MODE_U) {
                    *reinterpret_cast<float4 *>(A.xv + base + ib) = make_float4(xv[0], xv[1], xv[2], xv[3]);
                    *reinterpret_cast<float4 *>(A.zv + base + ib) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                }
                if (MODE == MODE_A)
                    *reinterpret_cast<float4 *>(A.out + base + ib) = make_float4(y[0], y[1], y[2], y[3]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pm[q] = pc[q];
                pc[q] = pn[q];
            }
            cm = cc;
            cc = cn;
        }
    }
    __syncthreads();
    if (s_abort) {
        if (threadIdx.x == 0 && MODE != MODE_A) {
            atomicExch(&A.st->status, 3);
            atomicExch(&A.st->done, 1);
        }
        if (MODE == MODE_A) return;
    }
    if (MODE == MODE_A) return;

    const int nb = gridDim.x * gridDim.y * gridDim.z;
    double t0, t1;
    if (MODE == MODE_P) {
        if (last_block_total<NTHREADS, false>(A.st, A.partials, nb, (double)acc0, 0.0, sred, t0, t1)) {
            if (threadIdx.x == 0) {
                CgState *s = A.st;
                s->sigma = t0;
                if (s->status == 3) {
                    s->done = 1;
                } else if (s->profile) {
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
        if (last_block_total<NTHREADS, true>(A.st, A.partials, nb, (double)acc0, (double)acc1, sred,
                                             t0, t1)) {
            if (threadIdx.x == 0) {
                CgState *s = A.st;
                s->beta = t0 / s->rho;
                s->rho = t0;
                s->rr = t1;
                s->iter += 1;
                if (s->status == 3) {
                    s->done = 1;
                } else if (s->profile) {
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
