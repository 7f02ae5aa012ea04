// FP32 PCG stencil kernels with TMA staging (included by solve.cu).
//
// Blocks are resident for the whole launch (one per resident slot) and pull
// work items -- z-chunks of KC planes of one 128 x 8 tile column -- from a
// global atomic counter.  The producer announces each chunk in a small
// descriptor ring before arming the chunk's first plane, so consumers learn
// it through the same mbarrier; the TMA pipeline keeps streaming across
// chunks.  One producer warp (lane 0) issues, for every plane, tensor-map
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
constexpr int NSLOT = 6;             // ring depth
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

// packed FP32 pairs (two independent lanes of arithmetic per instruction)
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}

}  // namespace tma

// MODE_P / MODE_U / MODE_A on the compressed FP32 operator.
template <int MODE>
__global__ void __launch_bounds__(tma::NTHREADS, 2)
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
    // work items: (tile column, z-chunk), chunks of one column consecutive
    const int xtiles = (g.nx - 1 + OWNW - 1) / OWNW;
    const int ytiles = (g.ny - 2 + ROWS - 1) / ROWS;
    const int nzi = g.nz - 2;
    const int nchunk = (nzi + A.KC - 1) / A.KC;
    const int nitems = xtiles * ytiles * nchunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NSLOT * L::stride);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSLOT);
    // descriptor ring (at most NSLOT chunks can be in flight)
    __shared__ int4 s_desc[NSLOT];

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, ROWS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();

    struct Seg {
        int i0, j0, kfirst, len;
    };
    auto decode = [&](int item) {
        Seg sg;
        const int col = item / nchunk, c = item - col * nchunk;
        sg.kfirst = 1 + c * A.KC;
        sg.len = min(A.KC, nzi - c * A.KC);
        sg.i0 = (col % xtiles) * OWNW;
        sg.j0 = 1 + (col / xtiles) * ROWS;
        return sg;
    };

    float acc0 = 0.f, acc1 = 0.f;
    if (w == ROWS) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            int last_use[NSLOT];
            for (int s = 0; s < NSLOT; ++s) last_use[s] = -1;
            int gt = 0, nseg = 0;  // running plane and chunk counters
            for (;;) {
                const int item = (int)atomicAdd(A.queue, 1u);
                const bool end = item >= nitems;
                const Seg sg = end ? Seg{0, 0, 0, -1} : decode(item);
                const int nplanes = end ? 1 : sg.len + 2;
                bool stop = false;
                for (int t = 0; t < nplanes; ++t, ++gt) {
                    const int s = gt % NSLOT, u = gt / NSLOT;
                    if (u > 0 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1)) {
                        s_abort = 1;
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)&s_abort) {
                        stop = true;
                        break;
                    }
                    const uint32_t bar = full0 + 8 * s;
                    if (t == 0) s_desc[nseg % NSLOT] = make_int4(sg.i0, sg.j0, sg.kfirst, sg.len);
                    if (end) {
                        mbar_arrive(bar);  // no data: announces the end
                        last_use[s] = -1;
                        break;
                    }
                    const uint32_t slot = smem_u32(smem + s * L::stride);
                    const int kp = sg.kfirst - 1 + t;
                    mbar_expect_tx(bar, L::tx);
                    tma_load3(slot + L::a, &maps.a, sg.i0 - 4, sg.j0 - 1, kp, bar);
                    if (MODE == MODE_P) tma_load3(slot + L::b, &maps.b, sg.i0 - 4, sg.j0 - 1, kp, bar);
                    if (MODE == MODE_U) {
                        tma_load3(slot + L::x, &maps.x, sg.i0, sg.j0, kp, bar);
                        tma_load3(slot + L::z, &maps.z, sg.i0, sg.j0, kp, bar);
                    }
                    tma_load3(slot + L::code, &maps.code, sg.i0 - 16, sg.j0 - 1, kp, bar);
                    last_use[s] = u;
                }
                ++nseg;
                if (end || stop) break;
            }
            // drain: every armed slot's copies must land before the block exits
            for (int s = 0; s < NSLOT; ++s)
                if (last_use[s] >= 0) mbar_wait(full0 + 8 * s, last_use[s] & 1);
        }
    } else {
        // ------------------------------------------------------- consumers
        const int r = w + 1;  // this row inside the halo boxes
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
        // streamed value (P: z + beta p_old) of box row rr
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

        int gt = 0, nseg = 0;
        bool ok = true;
        for (;; ++nseg) {
            // the chunk's first plane's barrier also publishes its descriptor
            if (!wait_full(gt)) {
                ok = false;
                break;
            }
            const int4 d = s_desc[nseg % NSLOT];
            if (d.w < 0) break;  // end of work
            const Seg sg{d.x, d.y, d.z, d.w};
            const int j = sg.j0 + w;
            const int ib = sg.i0 + lane * 4;
            const bool active = j <= g.ny - 2;
            const bool grp_ok = active && ib < g.sx;
            const int gt0 = gt;
            float pm[4], pc[4], pn[4];
            uint32_t cm = 0, cc = 0, cn = 0;
            // +z weights of this row at plane k-1 (the -z weights of plane k).
            // A plane on the fast path has no listed +z edge, so its pure +z
            // weights are exact too; only a segment's first plane loads them.
            float wzc[4] = {0.f, 0.f, 0.f, 0.f};
            {
                const uint8_t *s0 = slot_ptr(gt0);
                val4(s0, r, pm);
                cm = code4(s0, r);
                release(gt0);
                ok = wait_full(gt0 + 1);
            }
            if (ok) {
                const uint8_t *s1 = slot_ptr(gt0 + 1);
                val4(s1, r, pc);
                cc = code4(s1, r);
            }
            for (int t = 1; ok && t <= sg.len; ++t) {
                const int k = sg.kfirst + t - 1;
                if (!wait_full(gt0 + t + 1)) {
                    ok = false;
                    break;
                }
                const uint8_t *sc = slot_ptr(gt0 + t), *sn = slot_ptr(gt0 + t + 1);
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
                    // issue every listed-weight load first, then use them
                    const bool wz_valid = t > 1;
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
                if (fast) {
                    // packed: points (0,1) and (2,3) of this lane
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q0 = 2 * h;
                        const uint8_t ca = (uint8_t)(cc >> (8 * q0)), cb = (uint8_t)(cc >> (8 * q0 + 8));
                        const float2 x = f2(pc[q0], pc[q0 + 1]);
                        const float2 xl = f2(q0 == 0 ? left : pc[q0 - 1], pc[q0]);
                        const float2 xr = f2(pc[q0 + 1], q0 == 2 ? right : pc[q0 + 2]);
                        const float2 sum = __fadd2_rn(
                            __fadd2_rn(__fadd2_rn(sub2(x, xl), sub2(x, xr)),
                                       __fadd2_rn(sub2(x, f2(ym[q0], ym[q0 + 1])),
                                                  sub2(x, f2(yp[q0], yp[q0 + 1])))),
                            __fadd2_rn(sub2(x, f2(pm[q0], pm[q0 + 1])), sub2(x, f2(pn[q0], pn[q0 + 1]))));
                        const float2 wp = f2(wxp[q0], wxp[q0 + 1]);
                        const float2 kp = f2(cp.kappa(ca), cp.kappa(cb));
                        const float2 ap = __ffma2_rn(kp, x, __fmul2_rn(wp, sum));
                        const bool ia = grp_ok && ib + q0 >= 1 && ib + q0 <= g.nx - 2;
                        const bool ib2 = grp_ok && ib + q0 + 1 >= 1 && ib + q0 + 1 <= g.nx - 2;
                        if (MODE == MODE_P) {
                            // x is zero on boundary nodes, padding and absent rows
                            const float2 c = __fmul2_rn(x, ap);
                            acc0 += c.x + c.y;
                        } else if (MODE == MODE_U) {
                            const float2 dinv = f2((ca & 1) ? dinv_in : dinv_out, (cb & 1) ? dinv_in : dinv_out);
                            const float2 dg = f2((ca & 1) ? dg_in : dg_out, (cb & 1) ? dg_in : dg_out);
                            const float2 xn = __ffma2_rn(f2(alpha, alpha), x, f2(xv[q0], xv[q0 + 1]));
                            float2 zn = __ffma2_rn(__fmul2_rn(ap, dinv), f2(-alpha, -alpha),
                                                   f2(zv[q0], zv[q0 + 1]));
                            zn.x = ia ? zn.x : zv[q0];
                            zn.y = ib2 ? zn.y : zv[q0 + 1];
                            const float2 rr = __fmul2_rn(dg, zn);
                            const float2 c0 = __fmul2_rn(rr, zn), c1 = __fmul2_rn(rr, rr);
                            acc0 += c0.x + c0.y;
                            acc1 += c1.x + c1.y;
                            xv[q0] = xn.x;
                            xv[q0 + 1] = xn.y;
                            zv[q0] = zn.x;
                            zv[q0 + 1] = zn.y;
                        } else {
                            y[q0] = ia ? ap.x : 0.f;
                            y[q0 + 1] = ib2 ? ap.y : 0.f;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = ib + q;
                        const uint8_t c0 = (uint8_t)(cc >> (8 * q));
                        const float x0 = pc[q];
                        const float xl = q > 0 ? pc[q - 1] : left;
                        const float xr = q < 3 ? pc[q + 1] : right;
                        const float kp = cp.kappa(c0);
                        float ap = kp * x0;
                        ap += wxm[q] * (x0 - xl);
                        ap += wxp[q] * (x0 - xr);
                        ap += wym[q] * (x0 - ym[q]);
                        ap += wyp[q] * (x0 - yp[q]);
                        ap += wzm[q] * (x0 - pm[q]);
                        ap += wzp[q] * (x0 - pn[q]);
                        const float dg = ((((((wxm[q] + wxp[q]) + wym[q]) + wyp[q]) + wzm[q]) + wzp[q]) + kp);
                        const float dinv = 1.f / dg;
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
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) wzc[q] = wzp[q];
                release(gt0 + t);
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
            if (!ok) break;
            release(gt0 + sg.len + 1);  // the chunk's last plane (+z halo only)
            gt = gt0 + sg.len + 2;
        }
    }
    __syncthreads();
    // the last block to leave resets the work counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.queue + 1, 1u) == gridDim.x - 1) {
            A.queue[0] = 0u;
            A.queue[1] = 0u;
            __threadfence();
        }
    }
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
