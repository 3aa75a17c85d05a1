// Neural SDB in BF16 on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// f(p) = (|p| - r0 + alpha g(p)) / beta / lambda, g a ReLU MLP (the neural
// SDB of Sec. 5.2).  The W x W hidden layers run as tcgen05.mma GEMMs with
// BF16 operands and FP32 accumulation in tensor memory.  Layer 0 (3 -> W) is
// one K = 16 op per tile: the point's coordinates and the layer-0 weights
// split into BF16 high and low parts (x = x_h + x_l to 2^-17),
// A0 = [x_h x_l x_h  y_h y_l y_h  z_h z_l z_h  1 1  0 ...] against
// B0 = [wx_h wx_h wx_l  wy_h wy_h wy_l  wz_h wz_h wz_l  b_h b_l  0 ...], so that
// x_h wx_h + x_l wx_h + x_h wx_l and the bias are summed in FP32 (the omitted
// x_l wx_l is below 2^-16 of the term); its ReLU output is rounded to BF16 like
// every hidden activation.  The output layer (W -> 1) runs on CUDA cores in
// FP32.
//
// One persistent CTA per SM, 384 threads:
//   warp 0       TMA producer: 1-D bulk copies (cp.async.bulk) of BF16 weight
//                K-blocks, stored pre-swizzled in global memory, into a
//                2-stage shared-memory ring (mbarrier complete_tx).
//   warp 1       allocates TMEM; one lane issues tcgen05.mma for two 128-row
//                tiles per weight K-block (M = 128, N = W, K = 16 per op) and
//                tcgen05.commit's to the ring's "empty" barriers and to the
//                accumulator barrier.
//   warps 4..11  epilogue, one row (one ray or one point) per thread: layer 0,
//                TMEM -> registers (tcgen05.ld) -> bias, ReLU, BF16 -> the next
//                layer's A operand in 128B-swizzled K-major shared memory,
//                the FP32 output dot product, and the grid-hopping step of
//                Algorithm 1 (with the eps shrink) or the store of f.
// Every wait is bounded (2 s of %globaltimer); a timeout sets an error flag,
// makes all roles leave their loops, drains the copies in flight, and frees
// TMEM before the kernel returns.
#include <stdint.h>

#include "gh_internal.cuh"
#include "tc_ptx.cuh"

namespace gh {

namespace {

using namespace tc;

constexpr int EPI_T0 = 128;  // first epilogue thread (warp 4)
constexpr int TM = 128;      // rows per tile
constexpr int NSTAGE = 2;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr unsigned long long STOP_FLAGS = FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW;

enum { MODE_HOP = 0, MODE_VERTS = 1, MODE_POINTS = 2 };

// hidden layers supported by the tensor-core engine (at width 256 one fewer,
// for shared memory)
template <int W>
constexpr int maxmid_of() {
    return W == 256 ? 7 : 8;
}

template <int W>
struct SmemB {
    uint8_t a[2][W / 64][TM * 128];  // A operands: one per tile, K-blocks of 128 rows x 128 B (1024-aligned)
    uint8_t w[NSTAGE][W * 128];      // weight ring: one K-block of W rows x 128 B per stage
    uint8_t b0[2][W * 32];           // per tile: layer-0 operand B0 of its current item, W rows x 16 inputs
                                     // (32-byte swizzle: row n, 16-byte chunk c at (n/8)*256 + (n%8)*32 +
                                     // ((c ^ (n/4)%2) * 16))
    float bmid[2][maxmid_of<W>() * W];  // per tile: hidden-layer biases
    float zb[W];                        // zeros: the layer-0 phase adds no bias (B0 holds it)
    float wout[2][W];                // per tile: output-layer weights
    unsigned long long full[NSTAGE], empty[NSTAGE], acc_full[2], a_full[2], item_ready[2], drain;
    const uint16_t *cur_wbf[2];      // per tile: weights of its current item
    int done[2];                     // per tile: no more work
    uint32_t tmem_base;
    int ctl;
};

// OR-reduction over the 128 epilogue threads of one tile (named barrier id).
__device__ __forceinline__ bool epi_any(int id, bool v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ float outer_f(const MlpDev &m, float x, float y, float z, float g) {
    const float r = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    return (fmaf(m.alpha, g, m.radial * r - m.r0) / m.beta) * m.inv_lam;
}

// BF16 bits (round to nearest even) of x, and of the remainder x - bf16(x)
__device__ __forceinline__ void split2(float x, uint32_t &h, uint32_t &l) {
    uint32_t p;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(0.f), "f"(x));
    h = p & 0xFFFFu;
    const float r = x - __uint_as_float(h << 16);  // exact
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(p) : "f"(0.f), "f"(r));
    l = p & 0xFFFFu;
}

// Row o of tile t's layer-0 operand B0 (two 16-byte chunks, inputs 0..15).
template <int W>
__device__ __forceinline__ void put_b0(SmemB<W> &sm, int t, int o, float wx, float wy, float wz, float b) {
    uint32_t xh, xl, yh, yl, zh, zl, bh, bl;
    split2(wx, xh, xl);
    split2(wy, yh, yl);
    split2(wz, zh, zl);
    split2(b, bh, bl);
    const uint32_t base = su32(sm.b0[t]) + (uint32_t)((o >> 3) * 256 + (o & 7) * 32);
    const uint32_t sw = (uint32_t)((o >> 2) & 1);
    sts128(base + (sw << 4), xh | (xh << 16), xl | (yh << 16), yh | (yl << 16), zh | (zh << 16));
    sts128(base + ((1u ^ sw) << 4), zl | (bh << 16), bl, 0u, 0u);
}

// Item parameters of tile t (its 128 epilogue threads, or all threads at
// set-up with e and the stride given): B0, hidden biases, output weights.
template <int W>
__device__ __forceinline__ void load_item(SmemB<W> &sm, int t, const MlpDev &mm, int e, int stride) {
    for (int o = e; o < W; o += stride) {
        put_b0<W>(sm, t, o, mm.w0[3 * o], mm.w0[3 * o + 1], mm.w0[3 * o + 2], mm.b0[o]);
        sm.wout[t][o] = mm.wout[o];
    }
    for (int i = e; i < mm.n_mid * W; i += stride) sm.bmid[t][i] = mm.bm[i];
    fence_async_smem();  // B0 is read by the tensor core
}

// ---------------------------------------------------------------------------
// TILES 128-row tiles per CTA.  With two tiles the tensor core alternates
// between them (ping-pong): while tile 0's epilogue warps turn layer l into
// layer l+1's operand, the MMAs of tile 1's layer l run, and the other way
// round.  Each tile walks the items of the batch on its own: its rows take
// rays (or points) from item cur's queue, and when the item has no work left
// for the tile it moves to the next one, reloading its layer-0 weights,
// biases and output weights; the producer streams the weights of whichever
// item the phase's tile is on.
template <int W, int MODE, int TILES>
__global__ void __launch_bounds__(128 + 128 * TILES, 1)
    k_mlp_bf16(const Item *__restrict__ items, int n_items, const float *__restrict__ pts, long long npts,
               float *__restrict__ outv, unsigned long long wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    constexpr int KB = W / 64;
    constexpr int RS = KB < NSTAGE ? KB : NSTAGE;  // K-blocks a phase can take over from the one before
    constexpr uint32_t STAGE_BYTES = W * 128;
    constexpr uint32_t TMEM_COLS = TILES * W < 32 ? 32 : TILES * W;
    constexpr uint32_t IDESC = idesc_bf16(TM, W);
    SmemB<W> &sm = *reinterpret_cast<SmemB<W> *>(smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *ctl = &sm.ctl;
    Counters *ctr0 = items[0].s.ctr;  // error flags of a timeout go to the first item
    const int n_mid = items[0].m.n_mid;

    // ---- set-up ----------------------------------------------------------
    for (int t = 0; t < TILES; ++t) load_item<W>(sm, t, items[0].m, tid, blockDim.x);
    for (int i = tid; i < W; i += blockDim.x) sm.zb[i] = 0.f;
    if (tid == 0) {
        for (int i = 0; i < NSTAGE; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        for (int t = 0; t < 2; ++t) {
            mbar_init(&sm.acc_full[t], 1);
            mbar_init(&sm.a_full[t], 128);
            mbar_init(&sm.item_ready[t], 1);
            sm.cur_wbf[t] = items[0].m.wbf;
            sm.done[t] = t < TILES ? 0 : 1;
        }
        mbar_init(&sm.drain, 1);
        sm.ctl = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *vdone = sm.done;

    if (warp == 0) {
        // ---- TMA producer: the phases in the MMA's order ----------------------
        if (lane == 0) {
            long long issued = 0;
            int t = 0, lt[2] = {0, 0};
            bool fin[2] = {false, TILES < 2};
            uint32_t pir[2] = {0u, 0u};
            const uint8_t *src[2] = {nullptr, nullptr};
            bool go = true, keep = false;
            while (go && !(fin[0] && fin[1])) {
                if (fin[t]) {
                    t ^= 1;
                    continue;
                }
                if (lt[t] == 0) {  // a new step of tile t: its item (or its end) is decided first
                    if (!wait_bar(&sm.item_ready[t], pir[t], ctl, CTL_ABORT, ctr0, wait_ns)) break;
                    pir[t] ^= 1u;
                    if (vdone[t]) {
                        fin[t] = true;
                        if (!fin[t ^ 1]) t ^= 1;
                        continue;
                    }
                    src[t] = reinterpret_cast<const uint8_t *>(*(const uint16_t *volatile *)&sm.cur_wbf[t]);
                    // the layer-0 phase streams no weights
                    keep = false;
                    lt[t] = 1;
                    if (!fin[t ^ 1]) t ^= 1;
                    continue;
                }
                // A phase right after the other tile's phase of the same layer
                // of the same weights takes that phase's last RS K-blocks from
                // the ring (they are still there) and streams only the others.
                const bool reuse = keep;
                keep = !reuse && !fin[t ^ 1] && lt[t ^ 1] == lt[t] && src[t ^ 1] == src[t];
                for (int i = reuse ? RS : 0; i < KB; ++i) {
                    const int kb = reuse ? i - RS : i;
                    const int st = (int)(issued % NSTAGE);
                    const uint32_t par = (uint32_t)(((issued / NSTAGE) & 1) ^ 1);
                    if (!wait_bar(&sm.empty[st], par, ctl, CTL_ABORT, ctr0, wait_ns)) {
                        go = false;
                        break;
                    }
                    mbar_expect_tx(&sm.full[st], STAGE_BYTES);
                    bulk_g2s(sm.w[st], src[t] + (size_t)((lt[t] - 1) * KB + kb) * STAGE_BYTES, STAGE_BYTES,
                             &sm.full[st]);
                    ++issued;
                }
                lt[t] = lt[t] == n_mid ? 0 : lt[t] + 1;  // phases 0 (layer 0) .. n_mid (hidden layers)
                if (!fin[t ^ 1]) t ^= 1;
            }
            // the copies still in flight land before the CTA may exit
            for (long long i = issued - NSTAGE; i < issued; ++i) {
                if (i < 0) continue;
                wait_bar(&sm.full[i % NSTAGE], (uint32_t)((i / NSTAGE) & 1), ctl, 0, ctr0);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer: alternates between the tiles that still have work -----
        // The issuing thread is on the critical path (one tcgen05.mma takes
        // about 100 cycles to issue, a K = 16 op with N = 256 runs 128), so its
        // loop is kept lean: descriptors are built once and advanced by fixed
        // steps (K-blocks of A and ring stages are a fixed number of 16-byte
        // units apart, K = 16 is 2 units), a stage that has landed is taken
        // without a call, and the per-tile state lives in scalars.
        if (lane == 0) {
            long long consumed = 0;
            int t = 0, lt0 = 0, lt1 = 0;
            bool fin0 = false, fin1 = TILES < 2;
            uint32_t pa0 = 0u, pa1 = 0u;
            constexpr unsigned long long A_KB = (TM * 128) >> 4, W_ST = STAGE_BYTES >> 4;
            const unsigned long long ad0 = sdesc(su32(&sm.a[0][0][0])), ad1 = sdesc(su32(&sm.a[1][0][0]));
            const unsigned long long wd0 = sdesc(su32(sm.w[0]));
            const unsigned long long bd0 = sdesc32(su32(sm.b0[0])), bd1 = sdesc32(su32(sm.b0[1]));
            const uint16_t *w0 = nullptr, *w1 = nullptr;  // per tile: weights of its current item
            bool go = true, keep = false;
            while (go && !(fin0 && fin1)) {
                if (t ? fin1 : fin0) {
                    t ^= 1;
                    continue;
                }
                const uint32_t pa = t ? pa1 : pa0;
                if (!mbar_try(&sm.a_full[t], pa) && !wait_bar(&sm.a_full[t], pa, ctl, CTL_ABORT, ctr0, wait_ns)) break;
                if (t) pa1 ^= 1u;
                else pa0 ^= 1u;
                const int L = t ? lt1 : lt0;
                if (L == 0 && vdone[t]) {
                    if (t) fin1 = true;
                    else fin0 = true;
                    if (!(t ? fin0 : fin1)) t ^= 1;
                    continue;
                }
                if (L == 0) {
                    const uint16_t *w = *(const uint16_t *volatile *)&sm.cur_wbf[t];
                    if (t) w1 = w;
                    else w0 = w;
                }
                tc_fence_after();
                const unsigned long long ad = t ? ad1 : ad0;
                const uint32_t d = tmem + (uint32_t)(t * W);
                if (L == 0) {
                    // layer 0: A0 in the first 16 inputs of the A operand's K-block 0
                    umma(d, ad, t ? bd1 : bd0, IDESC, 0u);
                    keep = false;
                } else {
                    // the same rule as the producer: after the other tile's phase of
                    // this layer of the same weights, its last RS K-blocks (still in
                    // the ring) come first, then the K-blocks streamed for this phase
                    const bool reuse = keep;
                    keep = !reuse && !(t ? fin0 : fin1) && (t ? lt0 : lt1) == L && (t ? w0 : w1) == (t ? w1 : w0);
                    for (int i = 0; i < KB; ++i) {
                        int kb, st;
                        if (reuse && i < RS) {
                            kb = KB - RS + i;
                            st = (int)((consumed - RS + i) % NSTAGE);
                        } else {
                            kb = reuse ? i - RS : i;
                            st = (int)(consumed % NSTAGE);
                            const uint32_t par = (uint32_t)((consumed / NSTAGE) & 1);
                            if (!mbar_try(&sm.full[st], par) &&
                                !wait_bar(&sm.full[st], par, ctl, CTL_ABORT, ctr0, wait_ns)) {
                                go = false;
                                break;
                            }
                            ++consumed;
                        }
                        const unsigned long long a = ad + (unsigned long long)kb * A_KB;
                        const unsigned long long b = wd0 + (unsigned long long)st * W_ST;
                        umma(d, a, b, IDESC, i != 0);
                        umma(d, a + 2, b + 2, IDESC, 1u);
                        umma(d, a + 4, b + 4, IDESC, 1u);
                        umma(d, a + 6, b + 6, IDESC, 1u);
                        // a kept stage is released by the next phase, after its own use
                        if (!(keep && i >= KB - RS)) umma_commit(&sm.empty[st]);
                    }
                }
                if (!go) break;
                umma_commit(&sm.acc_full[t]);
                const int nl = L == n_mid ? 0 : L + 1;  // phases 0 (layer 0) .. n_mid (hidden layers)
                if (t) lt1 = nl;
                else lt0 = nl;
                if (!(t ? fin0 : fin1)) t ^= 1;
            }
            // every MMA issued above has completed before TMEM is released
            umma_commit(&sm.drain);
            wait_bar(&sm.drain, 0, ctl, 0, ctr0);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---- epilogue: one row per thread, 128 rows per tile -------------------
        const int t = (warp - 4) >> 2, row = tid - EPI_T0 - 128 * t, q = (warp - 4) & 3;
        const int bar = 1 + t;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(t * W);
        const uint32_t arow = su32(&sm.a[t][0][0]) + (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
        const int sw = row & 7;
        const unsigned lt = (1u << lane) - 1u;
        int cur = 0;
        const Item *it = &items[0];
        GridP g = it->g;  // the current item's grid and scratch, kept in registers
        Counters *ctr = it->s.ctr;
        unsigned long long *marks_raw = it->s.marks_raw;
        uint32_t *colcount = it->s.colcount;
        unsigned long long cap_marks = (unsigned long long)it->s.cap_marks;
        uint32_t col = NONE, rank = 0;
        int k = 0;
        bool done = false;
        float x = 0.f, y = 0.f;
        unsigned long long evals = 0, idx = 0;
        uint32_t pacc = 0;
        float *bmid = sm.bmid[t];
        float *wout = sm.wout[t];
        // a mark found in the previous step, written once its slot is known
        bool pend_mark = false;
        unsigned long long pend_base = 0, pend_rec = 0;
        unsigned pend_mask = 0;
        for (;;) {
            // 1. the work of this row, from item cur
            const int N = g.N;
            bool live = false;
            float px = 0.f, py = 0.f, pz = 0.f;
            if (MODE == MODE_HOP) {
                const uint32_t ncols = (uint32_t)N * (uint32_t)N;
                const bool need = col == NONE && !done;
                const unsigned needm = __ballot_sync(FULL, need);
                if (needm) {
                    const int leader = __ffs(needm) - 1;
                    unsigned long long base = 0;
                    if (lane == leader) base = atomicAdd(&ctr->next_col, (unsigned long long)__popc(needm));
                    base = __shfl_sync(FULL, base, leader);
                    if (need) {
                        const unsigned long long c = base + __popc(needm & lt);
                        if (c < ncols) {
                            col = column_of_claim((uint32_t)c, N);
                            k = 0;
                            rank = 0;
                            const int i = (int)(col / (uint32_t)N), j = (int)(col - (uint32_t)i * N);
                            x = fmaf((float)i + 0.5f, g.h, g.lo[0]);
                            y = fmaf((float)j + 0.5f, g.h, g.lo[1]);
                        } else {
                            done = true;
                        }
                    }
                }
                live = col != NONE;
                if (live) {
                    px = x;
                    py = y;
                    pz = fmaf((float)k + 0.5f, g.h, g.lo[2]);
                }
            } else {
                unsigned long long total = (unsigned long long)npts;
                if (MODE == MODE_VERTS)
                    total = (ctr->flags & STOP_FLAGS) ? 0ull : ctr->verts;
                unsigned long long base = 0;
                if (lane == 0) base = done ? total : atomicAdd(&ctr->next_tile, 32ull);
                base = __shfl_sync(FULL, base, 0);
                idx = base + lane;
                live = idx < total;
                if (base >= total) done = true;
                if (live) {
                    if (MODE == MODE_POINTS) {
                        px = pts[3 * idx];
                        py = pts[3 * idx + 1];
                        pz = pts[3 * idx + 2];
                    } else {
                        const unsigned long long key = it->s.vkey[idx];
                        const int N1 = N + 1;
                        const uint32_t line = (uint32_t)(key & 0xFFFFFFFFull), c = (uint32_t)(key >> 32);
                        const uint32_t a = line / (uint32_t)N1, b = line - a * (uint32_t)N1;
                        px = fmaf((float)a, g.h, g.lo[0]);
                        py = fmaf((float)b, g.h, g.lo[1]);
                        pz = fmaf((float)c, g.h, g.lo[2]);
                    }
                }
            }
            __syncwarp();
            const bool any = epi_any(bar, live);
            // the abort decision goes through the barrier so that it is uniform
            if (epi_any(bar, (*ctl & CTL_ABORT) != 0)) {
                if (row == 0) {
                    vdone[t] = 1;
                    __threadfence_block();
                    mbar_arrive(&sm.item_ready[t]);
                }
                mbar_arrive(&sm.a_full[t]);
                break;
            }
            if (!any) {
                // item cur has no work left for this tile: next item, or done
                if (MODE == MODE_HOP) {
                    if (pend_mark) {
                        const unsigned long long b0 = __shfl_sync(FULL, pend_base, __ffs(pend_mask) - 1);
                        if (pend_mask & (1u << lane)) {
                            const unsigned long long mi = b0 + __popc(pend_mask & lt);
                            if (mi < cap_marks) marks_raw[mi] = pend_rec;
                            else atomicOr(&ctr->flags, FLAG_MARK_OVERFLOW);
                        }
                    }
                    pend_mark = false;
                    pend_mask = 0;
                    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(FULL, evals, o);
                    if (lane == 0 && evals) atomicAdd(&ctr->hop_evals, evals);
                    evals = 0;
                }
                ++cur;
                if (cur >= n_items) {
                    if (row == 0) {
                        vdone[t] = 1;
                        __threadfence_block();
                        mbar_arrive(&sm.item_ready[t]);
                    }
                    mbar_arrive(&sm.a_full[t]);  // the tile's final phase: the MMA sees done
                    break;
                }
                it = &items[cur];
                g = it->g;
                ctr = it->s.ctr;
                marks_raw = it->s.marks_raw;
                colcount = it->s.colcount;
                cap_marks = (unsigned long long)it->s.cap_marks;
                col = NONE;
                done = false;
                load_item<W>(sm, t, it->m, row, 128);
                epi_any(bar, false);  // the new item's parameters are in place
                continue;
            }
            if (row == 0) {
                sm.cur_wbf[t] = it->m.wbf;
                mbar_arrive(&sm.item_ready[t]);
                if (MODE == MODE_HOP) atomicAdd(&ctr->row_slots, 128ull);
            }
            const MlpDev &m = it->m;
            // 2. the layer-0 operand A0 (BF16 high and low parts of the point, two
            // unit inputs for the bias) in the first 16 inputs of K-block 0
            {
                uint32_t xh, xl, yh, yl, zh, zl;
                split2(px, xh, xl);
                split2(py, yh, yl);
                split2(pz, zh, zl);
                constexpr uint32_t ONE = 0x3F80u;  // 1.0 in BF16
                sts128(arow + ((0 ^ sw) << 4), xh | (xl << 16), xh | (yh << 16), yl | (yh << 16), zh | (zl << 16));
                sts128(arow + ((1 ^ sw) << 4), zh | (ONE << 16), ONE, 0u, 0u);
            }
            fence_async_smem();
            mbar_arrive(&sm.a_full[t]);
            if (MODE == MODE_HOP && pend_mark) {
                // the previous step's marks: their slots came back meanwhile
                const unsigned long long b0 = __shfl_sync(FULL, pend_base, __ffs(pend_mask) - 1);
                if (pend_mask & (1u << lane)) {
                    const unsigned long long mi = b0 + __popc(pend_mask & lt);
                    if (mi < cap_marks) marks_raw[mi] = pend_rec;
                    else atomicOr(&ctr->flags, FLAG_MARK_OVERFLOW);
                }
                pend_mark = false;
                pend_mask = 0;
            }
            // 3. phases 0 (layer 0, its bias in B0) .. n_mid (hidden layers)
            float gsum = 0.f;
            for (int l = 0; l <= n_mid; ++l) {
                wait_bar(&sm.acc_full[t], pacc, ctl, CTL_ABORT, ctr0, wait_ns);
                pacc ^= 1u;
                __syncwarp();  // tcgen05.ld below needs the whole warp converged
                tc_fence_after();
                const float *bl = l ? bmid + (l - 1) * W : sm.zb;
                uint32_t ra[32], rb[32];
                tmem_ld32_async(taddr, ra);
                tmem_wait_ld();
                if (l < n_mid) {
#pragma unroll
                    for (int j = 0; j < W / 32; ++j) {
                        // the next chunk's load runs while this one is converted
                        uint32_t(&cu)[32] = (j & 1) ? rb : ra;
                        uint32_t(&nx)[32] = (j & 1) ? ra : rb;
                        if (j + 1 < W / 32) tmem_ld32_async(taddr + 32 * (j + 1), nx);
                        const float4 *bp = reinterpret_cast<const float4 *>(bl + 32 * j);
                        const int kb = j >> 1, c0 = (j & 1) * 4;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float4 b0 = bp[2 * c], b1 = bp[2 * c + 1];
                            const uint32_t p0 = pack_relu_bf16(__uint_as_float(cu[8 * c + 0]) + b0.x,
                                                               __uint_as_float(cu[8 * c + 1]) + b0.y);
                            const uint32_t p1 = pack_relu_bf16(__uint_as_float(cu[8 * c + 2]) + b0.z,
                                                               __uint_as_float(cu[8 * c + 3]) + b0.w);
                            const uint32_t p2 = pack_relu_bf16(__uint_as_float(cu[8 * c + 4]) + b1.x,
                                                               __uint_as_float(cu[8 * c + 5]) + b1.y);
                            const uint32_t p3 = pack_relu_bf16(__uint_as_float(cu[8 * c + 6]) + b1.z,
                                                               __uint_as_float(cu[8 * c + 7]) + b1.w);
                            sts128(arow + kb * (TM * 128) + (((c0 + c) ^ sw) << 4), p0, p1, p2, p3);
                        }
                        tmem_wait_ld();
                    }
                    tc_fence_before();
                    fence_async_smem();
                    mbar_arrive(&sm.a_full[t]);
                } else {
                    // output layer in FP32 from the accumulators
#pragma unroll
                    for (int j = 0; j < W / 32; ++j) {
                        uint32_t(&cu)[32] = (j & 1) ? rb : ra;
                        uint32_t(&nx)[32] = (j & 1) ? ra : rb;
                        if (j + 1 < W / 32) tmem_ld32_async(taddr + 32 * (j + 1), nx);
                        const float4 *bp = reinterpret_cast<const float4 *>(bl + 32 * j);
                        const float4 *wp = reinterpret_cast<const float4 *>(wout + 32 * j);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const float4 b = bp[c], w = wp[c];
                            gsum = fmaf(w.x, fmaxf(__uint_as_float(cu[4 * c + 0]) + b.x, 0.f), gsum);
                            gsum = fmaf(w.y, fmaxf(__uint_as_float(cu[4 * c + 1]) + b.y, 0.f), gsum);
                            gsum = fmaf(w.z, fmaxf(__uint_as_float(cu[4 * c + 2]) + b.z, 0.f), gsum);
                            gsum = fmaf(w.w, fmaxf(__uint_as_float(cu[4 * c + 3]) + b.w, 0.f), gsum);
                        }
                        tmem_wait_ld();
                    }
                    tc_fence_before();
                }
            }
            // 4. f, then the hop step or the store
            const float f = outer_f(m, px, py, pz, gsum + m.bout);
            if (MODE == MODE_HOP) {
                bool mark = false, empty = false;
                int step = 1;
                if (live) {
                    float d = fabsf(f) - g.eps;
                    if (!isfinite(f)) {
                        atomicOr(&ctr->flags, FLAG_NONFINITE);
                        d = 0.f;
                    }
                    if (d <= g.tau) {
                        mark = true;
                        empty = cell_is_empty(g, d, px, py, pz);
                    } else {
                        const float stp = floorf(d * g.inv_h);
                        step = stp < 1.f ? 1 : (stp > (float)N ? N : (int)stp);
                    }
                }
                const unsigned mm = __ballot_sync(FULL, mark);
                if (mm) {
                    // claim the slots now; the records are written after the next layer 0
                    const int leader = __ffs(mm) - 1;
                    if (lane == leader) pend_base = atomicAdd(&ctr->marks, (unsigned long long)__popc(mm));
                    pend_mark = true;
                    pend_mask = mm;
                    if (mark) pend_rec = pack_mark(col, (uint32_t)k, rank, empty);
                }
                if (live) {
                    if (mark) {
                        ++rank;
                        ++k;
                    } else {
                        k += step;
                    }
                    if (k >= N) {
                        colcount[col] = rank;
                        col = NONE;
                    }
                }
                if (live) ++evals;
            } else if (live) {
                if (MODE == MODE_VERTS) {
                    if (!isfinite(f)) atomicOr(&it->s.ctr->flags, FLAG_NONFINITE);
                    it->s.vval[idx] = f;
                } else {
                    outv[idx] = f;
                }
            }
        }
        (void)evals;
    }
    // ---- tear-down ---------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

template <int W, int MODE, int TILES>
void launch_bf16(const Item *items, int n_items, const float *p, long long n, float *out, int nsm, cudaStream_t st) {
    const size_t smem = sizeof(SmemB<W>) + 1024;
    cudaFuncSetAttribute(k_mlp_bf16<W, MODE, TILES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = nsm;
    if (MODE == MODE_POINTS) {
        const long long tiles = (n + 128 * TILES - 1) / (128 * TILES);
        if (grid > tiles) grid = (int)(tiles < 1 ? 1 : tiles);
    }
    k_mlp_bf16<W, MODE, TILES><<<grid, 128 + 128 * TILES, smem, st>>>(items, n_items, p, n, out, wait_limit_ns());
}

}  // namespace

#define GH_BF16_W(W, ...)                                     \
    switch (W) {                                              \
    case 64: { constexpr int WW = 64; __VA_ARGS__; } break;   \
    case 128: { constexpr int WW = 128; __VA_ARGS__; } break; \
    default: { constexpr int WW = 256; __VA_ARGS__; } break;  \
    }

bool bf16_supported(int width) { return width == 64 || width == 128 || width == 256; }
int bf16_max_mid(int width) { return width == 256 ? maxmid_of<256>() : maxmid_of<128>(); }

#define GH_BF16_T(T, ...)                                \
    if ((T) == 1) { constexpr int TT = 1; __VA_ARGS__; } \
    else { constexpr int TT = 2; __VA_ARGS__; }

void launch_hop_mlp_bf16(const Item *items, int n_items, int width, int nsm, int tiles, cudaStream_t st) {
    GH_BF16_W(width, GH_BF16_T(tiles, (launch_bf16<WW, MODE_HOP, TT>(items, n_items, nullptr, 0, nullptr, nsm, st))))
}

void launch_eval_vertices_mlp_bf16(const Item *items, int n_items, int width, int nsm, int tiles, cudaStream_t st) {
    GH_BF16_W(width,
              GH_BF16_T(tiles, (launch_bf16<WW, MODE_VERTS, TT>(items, n_items, nullptr, 0, nullptr, nsm, st))))
}

void launch_eval_points_mlp_bf16(const MlpDev &m, const float *p, long long n, float *out, int nsm,
                                 cudaStream_t st) {
    // one item whose counters live in a small private buffer
    static thread_local Counters *ctr = nullptr;
    static thread_local Item *ditem = nullptr;
    if (!ctr) cudaMalloc(&ctr, sizeof(Counters));
    if (!ditem) cudaMalloc(&ditem, sizeof(Item));
    Item h{};
    h.m = m;
    h.s.ctr = ctr;
    h.kind = 1;
    cudaMemsetAsync(ctr, 0, sizeof(Counters), st);
    cudaMemcpyAsync(ditem, &h, sizeof(Item), cudaMemcpyHostToDevice, st);
    GH_BF16_W(m.width, (launch_bf16<WW, MODE_POINTS, 2>(ditem, 1, p, n, out, nsm, st)))
}

}  // namespace gh
