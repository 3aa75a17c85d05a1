// Neural SDB on the tensor cores at FP32-level accuracy: split-BF16 products
// ("x6"), used for the refinement of the BF16 path and, through gh_eval, for
// point lists.
//
// Every FP32 operand x of a hidden layer is split exactly into three BF16
// parts, x = x_h + x_m + x_l (x_h = bf16(x), x_m = bf16(x - x_h), x_l =
// bf16(x - x_h - x_m); each difference is exact in FP32 and the three parts
// carry 24 significant bits).  Of the nine part products of a * w the six
// whose size is at least 2^-16 |a w| are formed on the tensor core (hh, hm,
// mh, hl, lh, mm) with FP32 accumulation in tensor memory; the three dropped
// (ml, lm, ll) are below 2^-23 |a w| together, the size of one FP32 rounding.
// Products are accumulated from the smallest to the largest: per layer the
// weight parts stream in the order low, middle, high, and within the high
// part's K-block the activation parts low, middle, high.  Layer 0 (3 -> W) and
// the output layer (W -> 1) run on CUDA cores in FP32, in the FP32 engine's
// operation order.
//
// One persistent CTA per SM, 384 threads, one 128-row tile at a time:
//   warp 0       bulk-copy producer: K-blocks (64 inputs x W outputs) of one
//                weight part per stage, stored pre-swizzled in global
//                memory, into a 4-stage shared-memory ring.
//   warp 1       allocates TMEM (2W columns); one lane issues tcgen05.mma
//                (M = 128, N = W, K = 16): A = x_h from shared memory, or
//                x_m / x_l from tensor memory.
//   warps 4..11  epilogue, two threads per row (column halves): layer 0,
//                TMEM -> registers -> bias, ReLU, the exact three-way split ->
//                x_h into 128B-swizzled shared memory and x_m, x_l into
//                tensor memory (the next layer's A operands); the output
//                dot product; the store of f.
// TMEM columns: [0, W) accumulator, [W, 3W/2) x_m, [3W/2, 2W) x_l (two BF16
// per 32-bit column, K ascending).  Every wait is bounded as in the BF16
// engine; a timeout sets the error flag, every role leaves, copies in flight
// land and MMAs complete before TMEM is freed.
#include <stdint.h>

#include "gh_internal.cuh"
#include "tc_ptx.cuh"

namespace gh {

namespace {

using namespace tc;

constexpr int TM = 128;   // rows per tile
constexpr int NST = 4;    // weight ring stages
constexpr int EPI = 256;  // epilogue threads (warps 4..11)
constexpr int MAXMID = 8;
constexpr unsigned long long STOP_FLAGS = FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW;
constexpr int BAR_EPI = 1;  // named barrier of the epilogue threads

enum { XMODE_REFINE = 0, XMODE_POINTS = 1 };

template <int W>
struct SmemX {
    uint8_t ah[W / 64][TM * 128];  // x_h: K-blocks of 128 rows x 128 B (1024-aligned)
    uint8_t w[NST][W * 128];       // weight ring: one K-block of one part per stage
    float4 w0b[W];                 // layer-0 rows and biases by output pairs (as the BF16 engine)
    float bmid[MAXMID * W];        // hidden-layer biases
    float wout[W];                 // output-layer weights
    float red[2][TM];              // output dot products of the two column halves
    unsigned long long full[NST], empty[NST], acc_full, a_full, item_ready, drain;
    const uint16_t *cur_w;         // split weights of the current item
    unsigned long long base, total;
    int done;
    uint32_t tmem_base;
    int ctl;
};

// x = h + m + l exactly, each part BF16 (rounded to nearest even); two values
// at a time, packed (lo value in the low half).
__device__ __forceinline__ void split3(float x0, float x1, uint32_t &h, uint32_t &m, uint32_t &l) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));
    const float r0 = x0 - __uint_as_float(h << 16), r1 = x1 - __uint_as_float(h & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(m) : "f"(r1), "f"(r0));
    const float s0 = r0 - __uint_as_float(m << 16), s1 = r1 - __uint_as_float(m & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(s1), "f"(s0));
}

__device__ __forceinline__ float outer_f(const MlpDev &m, float x, float y, float z, float g) {
    const float r = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    return (fmaf(m.alpha, g, m.radial * r - m.r0) / m.beta) * m.inv_lam;
}

// Loads item it's layer-0 rows, biases and output weights (epilogue threads).
template <int W>
__device__ __forceinline__ void load_params(SmemX<W> &sm, const MlpDev &mm, int e) {
    for (int o = e; o < W; o += EPI) {
        float *q = reinterpret_cast<float *>(&sm.w0b[o & ~1]) + (o & 1);
        q[0] = mm.w0[3 * o];
        q[2] = mm.w0[3 * o + 1];
        q[4] = mm.w0[3 * o + 2];
        q[6] = mm.b0[o];
        sm.wout[o] = mm.wout[o];
    }
    for (int i = e; i < mm.n_mid * W; i += EPI) sm.bmid[i] = mm.bm[i];
}

template <int W, int MODE>
__global__ void __launch_bounds__(384, 1)
    k_mlp_x6(const Item *__restrict__ items, int n_items, const float *__restrict__ pts, long long npts,
             float *__restrict__ outv, unsigned long long wait_ns) {
    extern __shared__ uint8_t smem_raw[];
    constexpr int KB = W / 64;                 // K-blocks per layer
    constexpr uint32_t STAGE_BYTES = W * 128;  // one K-block of one part
    constexpr uint32_t TMEM_COLS = 2 * W;      // 128, 256 or 512
    constexpr uint32_t AM = W, AL = W + W / 2; // TMEM columns of x_m and x_l
    constexpr uint32_t IDESC = idesc_bf16(TM, W);
    SmemX<W> &sm = *reinterpret_cast<SmemX<W> *>(smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *ctl = &sm.ctl;
    Counters *ctr0 = items[0].s.ctr;  // error flags of a timeout go to the first item
    const int n_mid = items[0].m.n_mid;

    if (tid >= 128) load_params<W>(sm, items[0].m, tid - 128);
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(&sm.acc_full, 1);
        mbar_init(&sm.a_full, EPI);
        mbar_init(&sm.item_ready, 1);
        mbar_init(&sm.drain, 1);
        sm.cur_w = items[0].m.wx6;
        sm.done = 0;
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
    volatile int *vdone = &sm.done;

    if (warp == 0) {
        // ---- producer: per tile, n_mid layers x 3 parts x KB K-blocks ----------
        if (lane == 0) {
            long long issued = 0;
            uint32_t pir = 0;
            bool go = true;
            while (go) {
                if (!wait_bar(&sm.item_ready, pir, ctl, CTL_ABORT, ctr0, wait_ns)) break;
                pir ^= 1u;
                if (*vdone) break;
                const uint8_t *src = reinterpret_cast<const uint8_t *>(*(const uint16_t *volatile *)&sm.cur_w);
                const int nst = n_mid * 3 * KB;
                for (int s = 0; s < nst; ++s) {
                    const int st = (int)(issued % NST);
                    const uint32_t par = (uint32_t)(((issued / NST) & 1) ^ 1);
                    if (!wait_bar(&sm.empty[st], par, ctl, CTL_ABORT, ctr0, wait_ns)) {
                        go = false;
                        break;
                    }
                    mbar_expect_tx(&sm.full[st], STAGE_BYTES);
                    bulk_g2s(sm.w[st], src + (size_t)s * STAGE_BYTES, STAGE_BYTES, &sm.full[st]);
                    ++issued;
                }
            }
            // the copies still in flight land before the CTA may exit
            for (long long i = issued - NST; i < issued; ++i) {
                if (i < 0) continue;
                wait_bar(&sm.full[i % NST], (uint32_t)((i / NST) & 1), ctl, 0, ctr0);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer ---------------------------------------------------------
        // (lean issue loop: descriptors built once and advanced by fixed steps,
        // a stage that has landed taken without a call; k_mlp_bf16.cu)
        if (lane == 0) {
            long long consumed = 0;
            uint32_t pa = 0;
            bool go = true;
            constexpr unsigned long long A_KB = (TM * 128) >> 4, W_ST = STAGE_BYTES >> 4;
            const unsigned long long ahd = sdesc(su32(&sm.ah[0][0])), wd0 = sdesc(su32(sm.w[0]));
            while (go) {
                for (int l = 0; l < n_mid && go; ++l) {
                    if (!wait_bar(&sm.a_full, pa, ctl, CTL_ABORT, ctr0, wait_ns)) {
                        go = false;
                        break;
                    }
                    pa ^= 1u;
                    if (l == 0 && *vdone) {
                        go = false;
                        break;
                    }
                    tc_fence_after();
                    for (int part = 0; part < 3 && go; ++part) {  // weight parts low, middle, high
                        for (int kb = 0; kb < KB; ++kb) {
                            const int st = (int)(consumed % NST);
                            const uint32_t par = (uint32_t)((consumed / NST) & 1);
                            if (!mbar_try(&sm.full[st], par) &&
                                !wait_bar(&sm.full[st], par, ctl, CTL_ABORT, ctr0, wait_ns)) {
                                go = false;
                                break;
                            }
                            const unsigned long long b0 = wd0 + (unsigned long long)st * W_ST;
                            const unsigned long long a0 = ahd + (unsigned long long)kb * A_KB;
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const unsigned long long bd = b0 + (unsigned long long)(2 * k);
                                const uint32_t acol = (uint32_t)(kb * 32 + k * 8);
                                if (part == 2) umma_ta(tmem, tmem + AL + acol, bd, IDESC, 1u);  // x_l w_h
                                if (part >= 1) umma_ta(tmem, tmem + AM + acol, bd, IDESC, 1u);  // x_m w_m, x_m w_h
                                umma(tmem, a0 + (unsigned long long)(2 * k), bd, IDESC,
                                     (part | kb | k) != 0);  // x_h w_l (the layer's first op), x_h w_m, x_h w_h
                            }
                            umma_commit(&sm.empty[st]);
                            ++consumed;
                        }
                    }
                    if (go) umma_commit(&sm.acc_full);
                }
            }
            // every MMA issued above has completed before TMEM is released
            umma_commit(&sm.drain);
            wait_bar(&sm.drain, 0, ctl, 0, ctr0);
        }
        __syncwarp();
    } else if (warp >= 4) {
        // ---- epilogue: two threads per row, column halves hf = 0, 1 --------------
        const int e = tid - 128, ew = e >> 5, q = ew & 3, hf = ew >> 2;
        const int row = 32 * q + lane;
        const uint32_t tlane = (uint32_t)(32 * q) << 16;
        const uint32_t arow = su32(&sm.ah[0][0]) + (uint32_t)((row >> 3) * 1024 + (row & 7) * 128);
        const int sw = row & 7;
        constexpr int HW = W / 2;  // columns (outputs, next-layer inputs) per thread
        int cur = 0;
        const Item *it = &items[0];
        uint32_t pacc = 0;
        for (;;) {
            // 1. the tile: 128 rows of item cur's list (or point array)
            if (e == 0) {
                unsigned long long total = (unsigned long long)npts, base = 0;
                if (MODE == XMODE_REFINE)
                    total = (it->s.ctr->flags & STOP_FLAGS) ? 0ull : it->s.ctr->refine;
                base = total ? atomicAdd(MODE == XMODE_REFINE ? &it->s.ctr->next_tile2 : &it->s.ctr->next_tile,
                                         (unsigned long long)TM)
                             : 0ull;
                sm.base = base;
                sm.total = total;
            }
            // the abort decision goes through the barrier so that it is uniform
            const bool abort = bar_any(BAR_EPI, EPI, (*ctl & CTL_ABORT) != 0);
            const unsigned long long base = sm.base, total = sm.total;
            if (abort || base >= total) {
                if (!abort && cur + 1 < n_items) {
                    // item cur has no rows left for this CTA: the next item
                    ++cur;
                    it = &items[cur];
                    load_params<W>(sm, it->m, e);
                    bar_sync(BAR_EPI, EPI);
                    continue;
                }
                if (e == 0) {
                    *vdone = 1;
                    __threadfence_block();
                    mbar_arrive(&sm.item_ready);
                }
                mbar_arrive(&sm.a_full);  // the final phase: the MMA sees done
                break;
            }
            if (e == 0) {
                sm.cur_w = it->m.wx6;
                mbar_arrive(&sm.item_ready);
            }
            const MlpDev &m = it->m;
            const GridP &g = it->g;
            const unsigned long long idx = base + (unsigned long long)row;
            const bool live = idx < total;
            float px = 0.f, py = 0.f, pz = 0.f;
            uint32_t vslot = 0;
            if (live) {
                if (MODE == XMODE_POINTS) {
                    px = pts[3 * idx];
                    py = pts[3 * idx + 1];
                    pz = pts[3 * idx + 2];
                } else {
                    vslot = it->s.rlist[idx];
                    const unsigned long long key = it->s.vkey[vslot];
                    const int N1 = g.N + 1;
                    const uint32_t line = (uint32_t)(key & 0xFFFFFFFFull), c = (uint32_t)(key >> 32);
                    const uint32_t a = line / (uint32_t)N1, b = line - a * (uint32_t)N1;
                    px = fmaf((float)a, g.h, g.lo[0]);
                    py = fmaf((float)b, g.h, g.lo[1]);
                    pz = fmaf((float)c, g.h, g.lo[2]);
                }
            }
            // 2. layer 0 in FP32 (the FP32 engine's operation order), split -> A operands
            __syncwarp();  // tcgen05.st below needs the whole warp converged
            {
                const unsigned long long ppx = pack2(px, px), ppy = pack2(py, py), ppz = pack2(pz, pz);
#pragma unroll 1
                for (int j = 0; j < HW / 32; ++j) {
                    const int c0 = hf * HW + 32 * j;  // first output of this 32-output chunk
                    uint32_t mh[16], ml[16], hh[16];
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const float4 wa = sm.w0b[c0 + 2 * p], wb = sm.w0b[c0 + 2 * p + 1];
                        const unsigned long long z = ffma2(pack2(wa.x, wa.y), ppx,
                                                           ffma2(pack2(wa.z, wa.w), ppy,
                                                                 ffma2(pack2(wb.x, wb.y), ppz, pack2(wb.z, wb.w))));
                        split3(fmaxf(lo2(z), 0.f), fmaxf(hi2(z), 0.f), hh[p], mh[p], ml[p]);
                    }
                    const int kb = c0 >> 6, cc = (c0 & 63) >> 3;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        sts128(arow + kb * (TM * 128) + (((cc + u) ^ sw) << 4), hh[4 * u], hh[4 * u + 1],
                               hh[4 * u + 2], hh[4 * u + 3]);
                    tmem_st16(tmem + tlane + AM + (uint32_t)(c0 / 2), mh);
                    tmem_st16(tmem + tlane + AL + (uint32_t)(c0 / 2), ml);
                }
                tmem_wait_st();
                tc_fence_before();
                fence_async_smem();
                mbar_arrive(&sm.a_full);
            }
            // 3. hidden layers: accumulator -> bias, ReLU -> split -> next A operands,
            //    and after the last one the output dot product
            float gs = 0.f;
            for (int l = 0; l < n_mid; ++l) {
                wait_bar(&sm.acc_full, pacc, ctl, CTL_ABORT, ctr0, wait_ns);
                pacc ^= 1u;
                __syncwarp();  // tcgen05.ld below needs the whole warp converged
                tc_fence_after();
                const float *bl = sm.bmid + l * W;
                const bool last = l + 1 == n_mid;
#pragma unroll 1
                for (int j = 0; j < HW / 32; ++j) {
                    const int c0 = hf * HW + 32 * j;
                    uint32_t acc[32];
                    tmem_ld32_async(tmem + tlane + (uint32_t)c0, acc);
                    tmem_wait_ld();
                    if (!last) {
                        uint32_t mh[16], ml[16], hh[16];
#pragma unroll
                        for (int p = 0; p < 16; ++p) {
                            const float2 b = *reinterpret_cast<const float2 *>(bl + c0 + 2 * p);
                            split3(fmaxf(__uint_as_float(acc[2 * p]) + b.x, 0.f),
                                   fmaxf(__uint_as_float(acc[2 * p + 1]) + b.y, 0.f), hh[p], mh[p], ml[p]);
                        }
                        const int kb = c0 >> 6, cc = (c0 & 63) >> 3;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            sts128(arow + kb * (TM * 128) + (((cc + u) ^ sw) << 4), hh[4 * u], hh[4 * u + 1],
                                   hh[4 * u + 2], hh[4 * u + 3]);
                        tmem_st16(tmem + tlane + AM + (uint32_t)(c0 / 2), mh);
                        tmem_st16(tmem + tlane + AL + (uint32_t)(c0 / 2), ml);
                    } else {
#pragma unroll
                        for (int p = 0; p < 32; ++p)
                            gs = fmaf(sm.wout[c0 + p], fmaxf(__uint_as_float(acc[p]) + bl[c0 + p], 0.f), gs);
                    }
                }
                if (!last) {
                    tmem_wait_st();
                    tc_fence_before();
                    fence_async_smem();
                    mbar_arrive(&sm.a_full);
                } else {
                    tc_fence_before();
                }
            }
            // 4. f = outer(g): the two halves' sums as the FP32 engine adds them
            sm.red[hf][row] = gs;
            bar_sync(BAR_EPI, EPI);
            if (hf == 0 && live) {
                const float g = sm.red[0][row] + sm.red[1][row] + m.bout;
                const float f = outer_f(m, px, py, pz, g);
                if (MODE == XMODE_REFINE) {
                    if (!isfinite(f)) atomicOr(&it->s.ctr->flags, FLAG_NONFINITE);
                    it->s.vval[vslot] = f;
                } else {
                    outv[idx] = f;
                }
            }
        }
    }
    // ---- tear-down ---------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

template <int W, int MODE>
void launch_x6(const Item *items, int n_items, const float *p, long long n, float *out, int nsm, cudaStream_t st) {
    const size_t smem = sizeof(SmemX<W>) + 1024;
    cudaFuncSetAttribute(k_mlp_x6<W, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = nsm;
    if (MODE == XMODE_POINTS) {
        const long long tiles = (n + TM - 1) / TM;
        if (grid > tiles) grid = (int)(tiles < 1 ? 1 : tiles);
    }
    k_mlp_x6<W, MODE><<<grid, 384, smem, st>>>(items, n_items, p, n, out, wait_limit_ns());
}

}  // namespace

#define GH_X6_W(W, ...)                                       \
    switch (W) {                                              \
    case 64: { constexpr int WW = 64; __VA_ARGS__; } break;   \
    case 128: { constexpr int WW = 128; __VA_ARGS__; } break; \
    default: { constexpr int WW = 256; __VA_ARGS__; } break;  \
    }

int x6_max_mid() { return MAXMID; }

void launch_refine_mlp_x6(const Item *items, int n_items, int width, int nsm, cudaStream_t st) {
    GH_X6_W(width, (launch_x6<WW, XMODE_REFINE>(items, n_items, nullptr, 0, nullptr, nsm, st)))
}

void launch_eval_points_mlp_x6(const MlpDev &m, const float *p, long long n, float *out, int nsm, cudaStream_t st) {
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
    GH_X6_W(m.width, (launch_x6<WW, XMODE_POINTS>(ditem, 1, p, n, out, nsm, st)))
}

}  // namespace gh
