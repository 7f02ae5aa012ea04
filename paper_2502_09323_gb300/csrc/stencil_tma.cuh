// FP32 PCG stencil kernels with TMA staging (included by solve.cu).
//
// One launch serves every system of a table (a single solve is a table of
// one; a batch of uneven solves is a table of many).  Blocks are resident for
// the whole launch and pull work items -- z-chunks of KC planes of one
// TW x (1024 / TW) tile column of one system (TW = 128, 64 or 32 per grid
// shape) -- from a global atomic counter.  The
// producer announces each chunk in a small descriptor ring before arming the
// chunk's first plane, so consumers learn it through the same mbarrier; the
// TMA pipeline keeps streaming across chunks and systems.
//
// One producer warp (lane 0) issues, for every plane, tensor-map
// (cp.async.bulk.tensor) loads of
//   * the streamed vector on a (TW + 8) x (TH + 2) box (4 columns of x halo
//     on each side and one halo row above and below; out-of-range elements
//     are zero), 136 x 10 for the 128 x 8 tile,
//   * for the update kernel, the x and z rows of the tile (TW x TH),
//   * the code bytes on a (TW + 32) x (TH + 2) box,
// into a ring of NSLOT shared-memory slots, each guarded by a "full" mbarrier
// (transaction bytes) and an "empty" mbarrier (one arrival per consumer warp).
// The 8 consumer warps compute TH / 8 rows each; a warp reads everything it
// needs from plane k's slot (its row, the rows above and below, the x-edge
// neighbours, codes) and releases it before it waits for plane k+1, keeping
// its own row of planes k-1, k, k+1 in registers, so the producer runs up to
// NSLOT-1 planes ahead of the slowest warp.  No consumer ever waits on
// another consumer.  Rows without listed edges take
// a packed FP32x2 fast path; rows with listed edges gather their weights,
// issued as soon as the plane's codes are at hand and before the warp waits
// for the next plane, so the gathers overlap that wait (the update kernel
// also prefetches the next plane's into L1).
//
// Dot products: each item's go to that item's own FP32 slot; the last block
// of the launch sums every system's slots in an order fixed by its item
// count (compensated FP32, FP64 for the total) and updates its CG state, so
// every result is independent of scheduling and of the other systems.
//
// A one-system launch may overlap the previous kernel of its stream
// (programmatic dependent launch): every read of data that kernel wrote
// comes after griddepcontrol.wait.
//
// Every wait is bounded: after g_slot_wait_limit polls (TMA_WAIT_LIMIT unless
// pb_set_wait_limit changed it) a slot wait gives up, the block records
// status 3 in the solver state, stops, waits (bounded by TMA_WAIT_LIMIT) for
// its own copies still in flight, and returns.
// Included inside solve.cu's anonymous namespace (needs KArgs, CoefC32,
// CgState and last_block_total from there).
#pragma once

namespace tma {

constexpr int ROWS = 8;              // consumer warps
constexpr int NSLOT = 6;             // ring depth
constexpr int NTHREADS = 32 * (ROWS + 1);
// A tile is TW x (1024 / TW) points of one plane (TW = 128, 64 or 32, chosen
// per grid shape): warp w owns tile rows w * RPW .. w * RPW + RPW - 1
// (RPW = 128 / TW rows per warp), TW / 4 lanes per row, 4 points a lane.
// Narrow tiles fit grids whose interior is not a multiple of 128 points
// across (97- or 161-node grids leave a quarter or three eighths of a
// 128-wide tile idle).  Boxes per plane:
//   streamed vector (TW + 8) x (TH + 2), x from i0 - 4, rows j0 - 1 .. j0 + TH
//   own rows        TW x TH, x from i0
//   code bytes      (TW + 32) x (TH + 2), x from i0 - 16
__host__ __device__ constexpr int tile_h(int tw) { return 1024 / tw; }
__host__ __device__ constexpr int box_w(int tw) { return tw + 8; }
__host__ __device__ constexpr int code_w(int tw) { return tw + 32; }
__host__ __device__ constexpr int box_h(int tw) { return 1024 / tw + 2; }
__host__ __device__ constexpr int box_bytes(int tw) { return box_w(tw) * box_h(tw) * 4; }
__host__ __device__ constexpr int code_bytes(int tw) { return code_w(tw) * box_h(tw); }
__host__ __device__ constexpr bool tile_ok(int tw) { return tw == 128 || tw == 64 || tw == 32; }
constexpr int TWDEF = 128;           // tile width unless tuned otherwise
constexpr long long TMA_WAIT_LIMIT = 1ll << 20;
// polls before a ring-slot wait (full or empty) gives up; the drain of the
// block's own copies at exit always uses TMA_WAIT_LIMIT
__device__ long long g_slot_wait_limit = TMA_WAIT_LIMIT;

constexpr int align128(int b) { return (b + 127) & ~127; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
// slot regions hold the largest box over the three tile widths
constexpr int BOX_BYTES = cmax(box_bytes(128), cmax(box_bytes(64), box_bytes(32)));      // 5440
constexpr int OWN_BYTES = 4096;                                                          // TW x TH floats
constexpr int CODE_BYTES = cmax(code_bytes(128), cmax(code_bytes(64), code_bytes(32)));  // 2176

// Slot regions hold the boxes of the tile width FIXW, or the largest over
// the three widths (FIXW = 0).
constexpr int box_region(int fixw) { return fixw ? box_bytes(fixw) : BOX_BYTES; }
constexpr int code_region(int fixw) { return fixw ? code_bytes(fixw) : CODE_BYTES; }

template <int MODE, int FIXW>
struct SlotLayout;
// direction kernel: z and p_old boxes + codes
template <int FIXW>
struct SlotLayout<0, FIXW> {
    static constexpr int a = 0, b = align128(box_region(FIXW)), x = -1, z = -1,
                         code = 2 * align128(box_region(FIXW));
    static constexpr int stride = align128(code + code_region(FIXW));
    __device__ static unsigned tx(int tw) { return 2 * box_bytes(tw) + code_bytes(tw); }
};
// update kernel: p box, x and z rows, codes
template <int FIXW>
struct SlotLayout<1, FIXW> {
    static constexpr int a = 0, b = -1, x = align128(box_region(FIXW)), z = x + OWN_BYTES,
                         code = z + OWN_BYTES;
    static constexpr int stride = align128(code + code_region(FIXW));
    __device__ static unsigned tx(int tw) { return box_bytes(tw) + 2 * OWN_BYTES + code_bytes(tw); }
};
// apply: x box + codes
template <int FIXW>
struct SlotLayout<2, FIXW> {
    static constexpr int a = 0, b = -1, x = -1, z = -1, code = align128(box_region(FIXW));
    static constexpr int stride = align128(code + code_region(FIXW));
    __device__ static unsigned tx(int tw) { return box_bytes(tw) + code_bytes(tw); }
};

template <int MODE, int FIXW>
constexpr int smem_bytes() {
    return NSLOT * SlotLayout<MODE, FIXW>::stride + 2 * NSLOT * 8;
}

struct Maps {  // boxes of the system's tile width TW (TH = 1024 / TW)
    CUtensorMap a;      // streamed vector, (TW + 8) x (TH + 2) box (P: z, U: p, A: x)
    CUtensorMap b;      // P: p_old, same box
    CUtensorMap x;      // U: x, TW x TH box
    CUtensorMap z;      // U: z, TW x TH box
    CUtensorMap code;   // (TW + 32) x (TH + 2) box of code bytes
};

// One system of a launch table (device memory).
struct SysEntry {  // aligned as CUtensorMap
    Maps P[2];          // direction kernel, p_old = pa (parity 0) / pb (1)
    Maps U[2];          // update kernel, p = pb (parity 0) / pa (1)
    Maps A;             // apply
    PadGeo pg;
    CoefC32 cp;
    float *pbuf[2];     // pa, pb
    float *x, *z;       // solution increment, preconditioned residual
    float *y;           // apply output
    CgState *st;
    float *partials;    // per item li: sigma at [li], rho and rr at
                        // [nitems + 2 li] and [nitems + 2 li + 1]
    unsigned int *cnt;  // items finished in the current launch
    int xtiles, ytiles, nchunk, KC, nitems, item_base;
    int tw;             // tile width (128, 64 or 32) of the maps and items
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
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false when the limit was reached (at once for limit 0).  Each
// poll may suspend the thread for up to 20 us until the phase completes (a
// waiting warp then issues no polling instructions; measured 1 % faster)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long n = 0; n < limit; ++n)
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

// the same load with an L2 cache policy (from createpolicy)
__device__ __forceinline__ void tma_load3h(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                           uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar), "l"(pol)
        : "memory");
}
// L2 policy: keep the lines (evicted last).  The code bytes (1 B per node,
// read by every launch of both kernels) take it, so they stay in L2 across
// launches while the streamed vectors pass through: measured U 79.7 -> 78.5
// us, P 69.9 -> 68.9 us at 257^3 (A/B on one box).  Giving the listed
// weights the same policy, or the vectors evict_first, was slower.
__device__ __forceinline__ uint64_t pol_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// packed FP32 pairs (two independent lanes of arithmetic per instruction)
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
// hint: bring the line holding p into L1 (no register result, no wait)
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// compensated FP32 sum (Neumaier): the value is s + c
__device__ __forceinline__ void nsum(float &s, float &c, float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
}
// the warp's compensated sums combined in a fixed tree (lane 0 holds them)
__device__ __forceinline__ void warp_nsum(float &s, float &c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        nsum(s, c, s2);
        c += c2;
    }
}

}  // namespace tma

// MODE_P / MODE_U / MODE_A on the compressed FP32 operator, over every
// system of tab (item_base ascending; total_items = sum of nitems).  With
// nsys < 0 the table size and item total are read from queue[2] and
// queue[3], so a captured launch follows a table that changes between
// replays.
// SINGLE: a launch over one system whose table entry (tensor maps,
// geometry, coefficients) is the kernel parameter e0, so that its values are
// read from the parameter bank instead of occupying registers; the
// arithmetic is the same as in the table form.
// FIXW: the tile width as a constant (every system of the launch has it),
// so that the lane and row indexing folds; 0 reads it per system.
template <int MODE, bool SINGLE, int FIXW>
__global__ void __launch_bounds__(tma::NTHREADS, 2)
k_stencil_tma(const tma::SysEntry *__restrict__ tab, int nsys, int total_items,
              unsigned int *queue, const __grid_constant__ tma::SysEntry e0) {
    using namespace tma;
    using L = SlotLayout<MODE, FIXW>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_abort, s_nsys, s_total, s_skip;
    __shared__ int s_desc[NSLOT][7];  // i0, j0, kfirst, len, system, local item, parity
    // per-descriptor warp partials of the dot products, combined without a
    // barrier: the warp that completes a descriptor's count sums them
    __shared__ float s_part[NSLOT][ROWS][2];
    __shared__ unsigned s_pcnt[NSLOT];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NSLOT * L::stride);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NSLOT);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSLOT; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, ROWS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        for (int q = 0; q < NSLOT; ++q) s_pcnt[q] = 0u;
    }
    // Programmatic dependent launch.  The set-up above touches only this
    // block's shared memory; the work counters, the CG state and the vectors
    // below are written by the previous kernel of the stream, so every thread
    // waits here for that kernel to complete (a no-op unless the launch asked
    // for programmatic serialization).  The next kernel may then be scheduled
    // as SMs free up; it waits the same way before touching our results.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const long long lim = g_slot_wait_limit;
    // A one-system launch issued after its solve finished (the host polls
    // with launches in flight) takes no work: the block skips to the exit
    // accounting below, so the last block still resets the work counters.
    // The flag is read once per block: a block of this launch whose wait
    // gives up sets it, so blocks that start later may see it set while
    // earlier ones took items; every block is still counted at the exit.
    if (threadIdx.x == 0) {
        s_skip = SINGLE && MODE != MODE_A && *(volatile int *)&e0.st->done;
        s_nsys = nsys < 0 ? (int)((volatile unsigned int *)queue)[2] : nsys;
        s_total = nsys < 0 ? (int)((volatile unsigned int *)queue)[3] : total_items;
    }
    __syncthreads();
    nsys = s_nsys;
    total_items = s_total;

    if (s_skip) {
        // no work: straight to the exit accounting
    } else if (w == ROWS) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            int last_use[NSLOT];
            for (int s = 0; s < NSLOT; ++s) last_use[s] = -1;
            const uint64_t keep = pol_last();
            int gt = 0, nseg = 0;  // running plane and chunk counters
            // a system's done flag and parity cannot change during this
            // launch before all its items are consumed (only its finaliser
            // changes them), so they are read once per system, not per item
            int csys = -1, cdone = 0, ccur = 0;
            for (;;) {
                const int item = (int)atomicAdd(queue, 1u);
                const bool end = item >= total_items;
                // The update kernel takes the items in reverse order: the
                // direction kernel before it wrote p in item order, so the p
                // of its last items is still in L2 when the update kernel
                // starts there, and the next direction kernel starts on the
                // z the update kernel wrote last.  Each item keeps its own
                // partial slot, so the sums do not depend on the order.
                const int it = MODE == MODE_U && !end ? total_items - 1 - item : item;
                int sys = 0, li = 0, i0 = 0, j0 = 0, kfirst = 0, len = -1, cur = 0, tw = TWDEF;
                const SysEntry *e = tab;
                if (!end) {
                    if constexpr (SINGLE) {
                        sys = 0;
                        e = &e0;
                    } else {
                        int lo = 0, hi = nsys - 1;  // last entry with item_base <= it
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (tab[mid].item_base <= it) lo = mid;
                            else hi = mid - 1;
                        }
                        sys = lo;
                        e = tab + sys;
                    }
                    if (MODE != MODE_A) {
                        if (sys != csys) {
                            cdone = *(volatile int *)&e->st->done;
                            ccur = *(volatile int *)&e->st->cur;
                            csys = sys;
                        }
                        if (cdone) continue;  // converged
                        cur = ccur;
                    }
                    li = it - e->item_base;
                    const int col = li / e->nchunk, c = li - col * e->nchunk;
                    kfirst = 1 + c * e->KC;
                    len = min(e->KC, e->pg.nz - 2 - c * e->KC);
                    tw = FIXW ? FIXW : e->tw;
                    i0 = (col % e->xtiles) * tw;
                    j0 = 1 + (col / e->xtiles) * tile_h(tw);
                }
                const Maps *m = MODE == MODE_P ? &e->P[cur] : (MODE == MODE_U ? &e->U[cur] : &e->A);
                const int nplanes = end ? 1 : len + 2;
                bool stop = false;
                for (int t = 0; t < nplanes; ++t, ++gt) {
                    const int s = gt % NSLOT, u = gt / NSLOT;
                    if (u > 0 && !mbar_wait(empty0 + 8 * s, (u - 1) & 1, lim)) {
                        s_abort = 1;
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)&s_abort) {
                        stop = true;
                        break;
                    }
                    const uint32_t bar = full0 + 8 * s;
                    if (t == 0) {
                        int *d = s_desc[nseg % NSLOT];
                        d[0] = i0;
                        d[1] = j0;
                        d[2] = kfirst;
                        d[3] = len;
                        d[4] = sys;
                        d[5] = li;
                        d[6] = cur;
                    }
                    if (end) {
                        mbar_arrive(bar);  // no data: announces the end
                        last_use[s] = -1;
                        break;
                    }
                    const uint32_t slot = smem_u32(smem + s * L::stride);
                    const int kp = kfirst - 1 + t;
                    mbar_expect_tx(bar, L::tx(tw));
                    tma_load3(slot + L::a, &m->a, i0 - 4, j0 - 1, kp, bar);
                    if constexpr (MODE == MODE_P) tma_load3(slot + L::b, &m->b, i0 - 4, j0 - 1, kp, bar);
                    if constexpr (MODE == MODE_U) {
                        tma_load3(slot + L::x, &m->x, i0, j0, kp, bar);
                        tma_load3(slot + L::z, &m->z, i0, j0, kp, bar);
                    }
                    tma_load3h(slot + L::code, &m->code, i0 - 16, j0 - 1, kp, bar, keep);
                    last_use[s] = u;
                }
                ++nseg;
                if (end || stop) break;
            }
            // drain: every armed slot's copies must land before the block exits
            for (int s = 0; s < NSLOT; ++s)
                if (last_use[s] >= 0) mbar_wait(full0 + 8 * s, last_use[s] & 1, TMA_WAIT_LIMIT);
        }
    } else {
        // ------------------------------------------------------- consumers
        // this lane's place in the tile, set per system from its tile width:
        // box row r (tile row r - 1), x lane xl of the row (the row's lanes
        // are 0 .. xlast), box and code row lengths bw and cw
        constexpr int TW0 = FIXW ? FIXW : TWDEF;
        constexpr int SH0 = TW0 == 128 ? 5 : (TW0 == 64 ? 4 : 3);  // log2(lanes per row)
        int tw = TW0, bw = box_w(TW0), cw = code_w(TW0), xl = lane & ((1 << SH0) - 1),
            xlast = (1 << SH0) - 1, r = 1 + w * (32 >> SH0) + (lane >> SH0);
        auto set_tile = [&](int t) {
            if (FIXW) return;
            const int sh = t == 128 ? 5 : (t == 64 ? 4 : 3);
            tw = t;
            bw = box_w(t);
            cw = code_w(t);
            xl = lane & ((1 << sh) - 1);
            xlast = (1 << sh) - 1;
            r = 1 + w * (32 >> sh) + (lane >> sh);
        };
        auto slot_ptr = [&](int t) { return smem + (t % NSLOT) * L::stride; };
        auto wait_full = [&](int t) -> bool {
            if (!mbar_wait(full0 + 8 * (t % NSLOT), (t / NSLOT) & 1, lim)) {
                s_abort = 1;
                return false;
            }
            return !*(volatile int *)&s_abort;
        };
        auto release = [&](int t) {
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * (t % NSLOT));
        };
        float beta = 0.f;
        // streamed value (P: z + beta p_old) of box row rr
        auto val4 = [&](const uint8_t *sl, int rr, float (&v)[4]) {
            const float *a = reinterpret_cast<const float *>(sl + L::a) + rr * bw + 4 + xl * 4;
            float4 t = *reinterpret_cast<const float4 *>(a);
            v[0] = t.x;
            v[1] = t.y;
            v[2] = t.z;
            v[3] = t.w;
            if (MODE == MODE_P) {
                const float *b = reinterpret_cast<const float *>(sl + L::b) + rr * bw + 4 + xl * 4;
                float4 u = *reinterpret_cast<const float4 *>(b);
                v[0] += beta * u.x;
                v[1] += beta * u.y;
                v[2] += beta * u.z;
                v[3] += beta * u.w;
            }
        };
        auto val1 = [&](const uint8_t *sl, int rr, int col) -> float {
            float v = reinterpret_cast<const float *>(sl + L::a)[rr * bw + col];
            if (MODE == MODE_P) v += beta * reinterpret_cast<const float *>(sl + L::b)[rr * bw + col];
            return v;
        };
        auto code4 = [&](const uint8_t *sl, int rr) -> uint32_t {
            return *reinterpret_cast<const uint32_t *>(sl + L::code + rr * cw + 16 + xl * 4);
        };

        int gt = 0, nseg = 0;
        // per-system values, reloaded only when the system changes (they
        // cannot change during the launch: finalisation runs at its end)
        int ksys = -1;
        PadGeo g{};
        CoefC32 cp{};
        float alpha = 0.f, dg_in = 0.f, dg_out = 0.f, dinv_in = 0.f, dinv_out = 0.f;
        float *pb0 = nullptr, *pb1 = nullptr, *yg = nullptr, *xg = nullptr, *zg = nullptr;
        if constexpr (SINGLE) {
            g = e0.pg;
            cp = e0.cp;
            if (MODE == MODE_P) beta = (float)e0.st->beta;
            if (MODE == MODE_U) alpha = (float)e0.st->alpha;
            dg_in = 6.f * cp.w_in;
            dg_out = 6.f * cp.w_out + cp.kap;
            dinv_in = 1.f / dg_in;
            dinv_out = 1.f / dg_out;
            pb0 = e0.pbuf[0];
            pb1 = e0.pbuf[1];
            yg = e0.y;
            xg = e0.x;
            zg = e0.z;
            set_tile(e0.tw);
            ksys = 0;
        }
        // Listed weights of this row at plane kp (codes in slot sl) go to L1
        // one plane before the slow path reads them, so that its gathers hit
        // L1 instead of waiting on DRAM (update kernel only: measured, it
        // shortens the update kernel and lengthens the direction kernel).  The addresses are exactly those the
        // slow path loads (own +x/+y/+z, the -y face from the row below, lane
        // 0's -x face, and the -z face from czb, the plane below's codes, when
        // its weights are not carried over from the previous plane); the
        // four points of a lane and face share one 16-byte run.
        auto prefetch_w = [&](const uint8_t *sl, int kp, int j, int ib, uint32_t cown,
                              uint32_t czb) {
            const uint32_t cyb = code4(sl, r - 1);
            const uint32_t lc = xl == 0 ? (uint32_t)sl[L::code + r * cw + 15] : 0u;
            const uint32_t need = (cown & 0x0E0E0E0Eu) | (cyb & 0x04040404u) |
                                  (czb & 0x08080808u) | (lc & 2u);
            if (!__any_sync(0xffffffffu, need != 0u)) return;
            const int pl = kp * (int)g.sxy + j * g.sx + ib;
            if (cown & 0x02020202u) prefetch_l1(cp.wx + pl);
            if (cown & 0x04040404u) prefetch_l1(cp.wy + pl);
            if (cown & 0x08080808u) prefetch_l1(cp.wz + pl);
            if (cyb & 0x04040404u) prefetch_l1(cp.wy + pl - g.sx);
            if (czb & 0x08080808u) prefetch_l1(cp.wz + pl - (int)g.sxy);
            if (lc & 2u) prefetch_l1(cp.wx + pl - 1);
        };
        for (;; ++nseg) {
            // the chunk's first plane's barrier also publishes its descriptor
            if (!wait_full(gt)) break;
            const int *d = s_desc[nseg % NSLOT];
            const int len = d[3];
            if (len < 0) break;  // end of work
            const int i0 = d[0], j0 = d[1], kfirst = d[2], sys = d[4], li = d[5], cur = d[6];
            const SysEntry *e = SINGLE ? &e0 : tab + sys;
            if (!SINGLE && sys != ksys) {
                g = e->pg;
                cp = e->cp;
                if (MODE == MODE_P) beta = (float)e->st->beta;
                if (MODE == MODE_U) alpha = (float)e->st->alpha;
                dg_in = 6.f * cp.w_in;
                dg_out = 6.f * cp.w_out + cp.kap;
                dinv_in = 1.f / dg_in;
                dinv_out = 1.f / dg_out;
                pb0 = e->pbuf[0];
                pb1 = e->pbuf[1];
                yg = e->y;
                xg = e->x;
                zg = e->z;
                set_tile(e->tw);
                ksys = sys;
            }
            float *const outp = MODE == MODE_P ? (cur ? pb0 : pb1) : (MODE == MODE_A ? yg : nullptr);
            const int j = j0 + r - 1;
            const int ib = i0 + xl * 4;
            const bool active = j <= g.ny - 2;
            const bool grp_ok = active && ib < g.sx;
            const int gt0 = gt;
            float acc0 = 0.f, acc1 = 0.f;
            float pm[4], pc[4], pn[4];
            uint32_t cm = 0, cc = 0, cn = 0;
            // +z weights of this row at plane k-1 (the -z weights of plane k).
            // A plane on the fast path has no listed +z edge, so its pure +z
            // weights are exact too; only a chunk's first plane loads them.
            float wzc[4] = {0.f, 0.f, 0.f, 0.f};
            bool ok = true;
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
                if (MODE == MODE_U) prefetch_w(s1, kfirst, j, ib, cc, cm);
            }
            for (int t = 1; ok && t <= len; ++t) {
                const int k = kfirst + t - 1;
                const uint8_t *sc = slot_ptr(gt0 + t), *sn = slot_ptr(gt0 + t + 1);
                // plane t's codes are all here (its slot is full): decide the
                // path and issue the listed-weight gathers first, so that they
                // are in flight while this warp waits for plane t+1
                const uint32_t cym = code4(sc, r - 1);
                const uint32_t lcode = sc[L::code + r * cw + 15 + xl * 4];
                const uint32_t cxl = (cc << 8) | lcode;
                const uint32_t special = (cc & 0x0E0E0E0Eu) | (cxl & 0x02020202u) |
                                         (cym & 0x04040404u) | (cm & 0x08080808u);
                const bool fast = !__any_sync(0xffffffffu, special != 0u);
                const int base = k * (int)g.sxy + j * g.sx;
                // per-point weights of the six faces
                float wxp[4], wxm[4], wyp[4], wym[4], wzp[4], wzm[4];
                float wl = 0.f;
                if (fast) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float wp = cp.pure((uint8_t)(cc >> (8 * q)));
                        wxp[q] = wxm[q] = wyp[q] = wym[q] = wzp[q] = wzm[q] = wp;
                    }
                } else {
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
                    if (xl == 0) wl = (lcode & 2) ? __ldg(cp.wx + pl - 1) : cp.pure((uint8_t)cc);
                }
                float ym[4], yp[4];
                val4(sc, r - 1, ym);
                val4(sc, r + 1, yp);
                float left = __shfl_up_sync(0xffffffffu, pc[3], 1);
                float right = __shfl_down_sync(0xffffffffu, pc[0], 1);
                if (xl == 0) left = val1(sc, r, 3);
                if (xl == xlast) right = val1(sc, r, 4 + tw);
                float xv[4] = {0.f, 0.f, 0.f, 0.f}, zv[4] = {0.f, 0.f, 0.f, 0.f};
                if (MODE == MODE_U) {
                    float4 a = *reinterpret_cast<const float4 *>(sc + L::x + ((r - 1) * tw + xl * 4) * 4);
                    float4 b = *reinterpret_cast<const float4 *>(sc + L::z + ((r - 1) * tw + xl * 4) * 4);
                    xv[0] = a.x;
                    xv[1] = a.y;
                    xv[2] = a.z;
                    xv[3] = a.w;
                    zv[0] = b.x;
                    zv[1] = b.y;
                    zv[2] = b.z;
                    zv[3] = b.w;
                }
                // every read of plane t's slot is done: release it before waiting
                // for plane t+1, so a warp holds one slot at a time
                release(gt0 + t);
                if (!wait_full(gt0 + t + 1)) {
                    ok = false;
                    break;
                }
                val4(sn, r, pn);
                cn = code4(sn, r);
                if (MODE == MODE_U && t < len) prefetch_w(sn, k + 1, j, ib, cn, 0u);
                if (!fast) {
                    // -x weight of point q is the +x weight of point q-1
                    const float wsh = __shfl_up_sync(0xffffffffu, wxp[3], 1);
                    wxm[0] = xl == 0 ? wl : wsh;
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
                    // per-point weights, packed like the fast path: points
                    // (0,1) and (2,3) of this lane, each FP32x2 step rounding
                    // as the scalar expression it stands for
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int q0 = 2 * h;
                        const uint8_t ca = (uint8_t)(cc >> (8 * q0)), cb = (uint8_t)(cc >> (8 * q0 + 8));
                        const float2 x = f2(pc[q0], pc[q0 + 1]);
                        const float2 xl = f2(q0 == 0 ? left : pc[q0 - 1], pc[q0]);
                        const float2 xr = f2(pc[q0 + 1], q0 == 2 ? right : pc[q0 + 2]);
                        const float2 kp = f2(cp.kappa(ca), cp.kappa(cb));
                        const float2 w0 = f2(wxm[q0], wxm[q0 + 1]), w1 = f2(wxp[q0], wxp[q0 + 1]);
                        const float2 w2 = f2(wym[q0], wym[q0 + 1]), w3 = f2(wyp[q0], wyp[q0 + 1]);
                        const float2 w4 = f2(wzm[q0], wzm[q0 + 1]), w5 = f2(wzp[q0], wzp[q0 + 1]);
                        float2 ap = __fmul2_rn(kp, x);
                        ap = __ffma2_rn(w0, sub2(x, xl), ap);
                        ap = __ffma2_rn(w1, sub2(x, xr), ap);
                        ap = __ffma2_rn(w2, sub2(x, f2(ym[q0], ym[q0 + 1])), ap);
                        ap = __ffma2_rn(w3, sub2(x, f2(yp[q0], yp[q0 + 1])), ap);
                        ap = __ffma2_rn(w4, sub2(x, f2(pm[q0], pm[q0 + 1])), ap);
                        ap = __ffma2_rn(w5, sub2(x, f2(pn[q0], pn[q0 + 1])), ap);
                        const bool ia = grp_ok && ib + q0 >= 1 && ib + q0 <= g.nx - 2;
                        const bool ib2 = grp_ok && ib + q0 + 1 >= 1 && ib + q0 + 1 <= g.nx - 2;
                        if (MODE == MODE_P) {
                            const float2 c = __fmul2_rn(x, ap);
                            if (ia) acc0 += c.x;
                            if (ib2) acc0 += c.y;
                        } else if (MODE == MODE_U) {
                            const float2 dg = __fadd2_rn(
                                __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(w0, w1), w2), w3), w4), w5),
                                kp);
                            // hardware reciprocal (about 1 ulp): a Jacobi scale inside the FP32 solve
                            const float2 ndinv = f2(-__fdividef(1.f, dg.x), -__fdividef(1.f, dg.y));
                            const float2 xn = __ffma2_rn(f2(alpha, alpha), x, f2(xv[q0], xv[q0 + 1]));
                            const float2 zn = __ffma2_rn(__fmul2_rn(f2(alpha, alpha), ap), ndinv,
                                                         f2(zv[q0], zv[q0 + 1]));
                            const float2 rr = __fmul2_rn(dg, zn);
                            const float2 c0 = __fmul2_rn(rr, zn), c1 = __fmul2_rn(rr, rr);
                            if (ia) {
                                xv[q0] = xn.x;
                                zv[q0] = zn.x;
                                acc0 += c0.x;
                                acc1 += c1.x;
                            }
                            if (ib2) {
                                xv[q0 + 1] = xn.y;
                                zv[q0 + 1] = zn.y;
                                acc0 += c0.y;
                                acc1 += c1.y;
                            }
                        } else {
                            y[q0] = ia ? ap.x : 0.f;
                            y[q0 + 1] = ib2 ? ap.y : 0.f;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) wzc[q] = wzp[q];
                if (grp_ok) {
                    if (MODE == MODE_P)
                        *reinterpret_cast<float4 *>(outp + base + ib) = make_float4(pc[0], pc[1], pc[2], pc[3]);
                    if (MODE == MODE_U) {
                        *reinterpret_cast<float4 *>(xg + base + ib) = make_float4(xv[0], xv[1], xv[2], xv[3]);
                        *reinterpret_cast<float4 *>(zg + base + ib) = make_float4(zv[0], zv[1], zv[2], zv[3]);
                    }
                    if (MODE == MODE_A)
                        *reinterpret_cast<float4 *>(outp + base + ib) = make_float4(y[0], y[1], y[2], y[3]);
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
            release(gt0 + len + 1);  // the chunk's last plane (+z halo only)
            gt = gt0 + len + 2;
            if (MODE == MODE_A) continue;

            // ---- dot products of this item: the 8 row warps combine their
            // partials in shared memory (the warp that completes the count
            // sums them in row order) and that warp stores the item's partial.
            // The last block of the launch sums each system's item partials
            // in item order and updates its CG state.  No warp waits for
            // another.
            // (FP32 across the warp: the FP64 pipe of this part is narrow)
            const float b0 = warp_sum_f(acc0), b1 = warp_sum_f(acc1);
            const int ps = nseg % NSLOT;
            if (lane == 0) {
                s_part[ps][w][0] = b0;
                s_part[ps][w][1] = b1;
                __threadfence_block();
                if (atomicAdd(&s_pcnt[ps], 1u) == (unsigned)ROWS - 1) {
                    __threadfence_block();
                    float t0 = 0.f, t1 = 0.f;
                    for (int r = 0; r < ROWS; ++r) {
                        t0 += *(volatile float *)&s_part[ps][r][0];
                        t1 += *(volatile float *)&s_part[ps][r][1];
                    }
                    s_pcnt[ps] = 0u;
                    const int nit = e->nitems;
                    if (MODE == MODE_P) {
                        e->partials[li] = t0;
                    } else {
                        e->partials[nit + 2 * li] = t0;
                        e->partials[nit + 2 * li + 1] = t1;
                    }
                }
            }
        }
    }
    // this thread's item partials are visible device-wide before the block
    // counts itself done
    __threadfence();
    __syncthreads();
    // a device-side wait gave up: stop every system of the table
    if (s_abort && threadIdx.x == 0 && MODE != MODE_A) {
        for (int q = 0; q < nsys; ++q) {
            atomicExch(&tab[q].st->status, 3);
            atomicExch(&tab[q].st->done, 1);
        }
    }
    // the last block to leave finishes every system's reductions and resets
    // the work counters for the next launch
    __shared__ int s_lastblk;
    if (threadIdx.x == 0) {
        __threadfence();
        s_lastblk = atomicAdd(queue + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_lastblk) return;
    __threadfence();
    if (MODE != MODE_A) {
        // Each system's item partials are summed in an order fixed by its
        // item count only: systems of more than BIGSYS items by the whole
        // block (thread t takes items t, t+NTHREADS, ...), smaller ones by
        // one warp each.  The sums are compensated FP32 up to the warps'
        // totals (this block runs alone at the end of the launch, on the
        // critical path, and FP64 is a narrow pipe of GB300) and FP64 after.
        constexpr int BIGSYS = 512;
        __shared__ double s_red[2][NTHREADS / 32];
        auto finish = [&](CgState *st, double t0, double t1) {
            if (st->split) {
                // one slab of a split solve: its totals only
                st->part0 = t0;
                st->part1 = t1;
                return;
            }
            if (MODE == MODE_P) {
                st->sigma = t0;
                if (st->status == 3) {
                    st->done = 1;
                } else if (st->profile) {
                    st->alpha = isfinite(t0) && t0 != 0.0 ? st->rho / t0 : 0.0;
                } else if (!(t0 > 0.0) || !isfinite(t0)) {
                    st->done = 1;
                    st->status = 1;
                } else {
                    st->alpha = st->rho / t0;
                }
            } else {
                st->beta = t0 / st->rho;
                st->rho = t0;
                st->rr = t1;
                st->iter += 1;
                st->cur ^= 1;  // the new p_old is this iteration's p
                if (st->status == 3) {
                    st->done = 1;
                } else if (st->profile) {
                    // timing run: keep going
                } else if (!isfinite(t1)) {
                    st->done = 1;
                    st->status = 1;
                } else if (t1 <= st->rr_stop) {
                    st->done = 1;
                    st->status = 0;
                } else if (st->iter >= st->max_iter) {
                    st->done = 1;
                    st->status = 2;
                }
            }
        };
        // the warp's items summed; the totals are valid in lane 0
        auto item_sums = [&](const SysEntry *e, int first, int stride, double &t0, double &t1) {
            const int nit = e->nitems;
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
#pragma unroll 4
            for (int i = first; i < nit; i += stride) {
                if (MODE == MODE_P) {
                    nsum(s0, c0, __ldcg(e->partials + i));
                } else {
                    nsum(s0, c0, __ldcg(e->partials + nit + 2 * i));
                    nsum(s1, c1, __ldcg(e->partials + nit + 2 * i + 1));
                }
            }
            warp_nsum(s0, c0);
            if (MODE != MODE_P) warp_nsum(s1, c1);
            t0 = (double)s0 + (double)c0;
            t1 = (double)s1 + (double)c1;
        };
        // large systems: the whole block, one after the other
        for (int q = 0; q < nsys; ++q) {
            const SysEntry *e = tab + q;
            const int nit = e->nitems;
            if (nit <= BIGSYS || *(volatile int *)&e->st->done) continue;
            double t0, t1;
            item_sums(e, threadIdx.x, NTHREADS, t0, t1);
            if (lane == 0) {
                s_red[0][w] = t0;
                s_red[1][w] = t1;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double u0 = 0.0, u1 = 0.0;
                for (int r = 0; r < NTHREADS / 32; ++r) {
                    u0 += s_red[0][r];
                    u1 += s_red[1][r];
                }
                finish(e->st, u0, u1);
            }
            __syncthreads();
        }
        // small systems: one warp each
        for (int q = w; q < nsys; q += NTHREADS / 32) {
            const SysEntry *e = tab + q;
            const int nit = e->nitems;
            CgState *st = e->st;
            // systems that were done at launch (or stopped by an abort) have no partials
            if (nit == 0 || nit > BIGSYS || *(volatile int *)&st->done) continue;
            double t0, t1;
            item_sums(e, lane, 32, t0, t1);
            if (lane == 0) finish(st, t0, t1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        queue[0] = 0u;
        queue[1] = 0u;
        __threadfence();
    }
}
