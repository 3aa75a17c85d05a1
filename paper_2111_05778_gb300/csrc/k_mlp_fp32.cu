// Neural SDB in FP32 on the FFMA pipe.
//
// f(p) = (|p| - r0 + alpha g(p)) / beta / lambda with g a ReLU MLP (the
// neural SDB of Sec. 5.2, Eq. 7).  A CTA of 256 threads evaluates a tile of
// 128 points at a time: layer 0 (3 -> W) and the output layer (W -> 1) on
// CUDA cores directly, the W x W hidden layers as register-blocked FP32
// products (8 rows x W/16 outputs per thread) whose weights stream from L2
// through a two-buffer shared-memory ring: one thread issues each 32-row
// chunk as a 1-D bulk copy (cp.async.bulk, mbarrier complete_tx), every warp
// waits for the chunk on its own, and the last warp to finish reading a
// buffer issues the chunk two ahead into it -- the warps drift freely inside
// a layer and meet only around the activation write-back at its end.
//
// Two users of the tile engine:
//   k_hop_mlp_fp32   persistent grid hopper: each of the 128 rows is a ray;
//                    after every tile the ray marks / jumps (Algorithm 1) and
//                    dead rows are refilled from the column queue.
//   k_pts_mlp_fp32   a list of points (lattice vertices of marked cells, or
//                    an explicit point array).
#include "gh_internal.cuh"

namespace gh {

namespace {

constexpr int TM = 128;   // rows per tile
constexpr int KC = 32;    // K rows per weight chunk
constexpr int NT = 256;   // threads per CTA
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr unsigned long long STOP_FLAGS = FLAG_MARK_OVERFLOW | FLAG_VERT_OVERFLOW;

constexpr unsigned long long WAIT_NS = 2000000000ull;

template <int W>
struct Smem {
    float act[W][TM + 4];  // activations, feature-major
    float wbuf[2][KC * W]; // weight chunk ring
    float4 p[TM];          // query points
    float g[TM];           // network output
    float red[TM];
    unsigned long long full[2];  // chunk landed in buffer b (complete_tx)
    unsigned int done[2];        // warps finished with buffer b
    int abort;                   // a chunk wait gave up after 2 s: stop waiting
    unsigned long long wait_ns;  // the caller's wait limit (gh_set_wait_limit_ns)
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity of buffer b's barrier.  What it
// waits for is one of this CTA's own bulk copies, which lands: at the caller's
// limit (sm.wait_ns) the timeout is recorded in the device flags and the wait
// goes on, so that no copy is ever left in flight; only after 2 s does it set
// the abort bit (later waits return at once) and return.
template <int W>
__device__ __noinline__ void wait_chunk(Smem<W> &sm, int b, uint32_t parity, Counters *ctr) {
    const unsigned long long lim = sm.wait_ns;
    bool flagged = false;
    if (lim == 0) {  // a limit of 0: the wait counts as run out at once (the timeout path's test device)
        atomicOr(&ctr->flags, FLAG_TIMEOUT);
        flagged = true;
    }
    if (mbar_try(&sm.full[b], parity)) return;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(&sm.full[b], parity)) return;
        if (*(volatile int *)&sm.abort) return;
        if ((it & 255) == 0 || lim < 100000ull) {
            const unsigned long long dt = gtimer() - t0;
            if (!flagged && dt > lim) {
                atomicOr(&ctr->flags, FLAG_TIMEOUT);
                flagged = true;
            }
            if (dt > WAIT_NS) {
                atomicOr((int *)&sm.abort, 1);
                atomicOr(&ctr->flags, FLAG_TIMEOUT);
                return;
            }
        }
    }
}

// What a tile pass computes: the network value (EVAL), the same with every
// layer's pre-activation stored (FWDZ, the adjoint's forward pass), or the
// adjoint's delta chain delta_{l-1} = (W_l^T delta_l) * [z_{l-1} > 0] from
// delta_L down to delta_0, every delta stored (BACK).
enum { EVAL = 0, FWDZ = 1, BACK = 2 };

// chunk ch of the hidden layers (K rows ch*KC.. of the pass's ch/NCH-th
// layer: layer ch/NCH of wt, or for BACK layer n_mid-1-ch/NCH of wtb) into
// buffer b
template <int W, int KIND>
__device__ __forceinline__ void issue_chunk(const MlpDev &m, Smem<W> &sm, int ch, int b) {
    constexpr int NCH = W / KC;
    constexpr uint32_t BYTES = KC * W * 4;
    const int l = ch / NCH, c = ch - l * NCH;
    const float *src = (KIND == BACK ? m.wtb + (size_t)(m.n_mid - 1 - l) * W * W : m.wt + (size_t)l * W * W) +
                       (size_t)c * KC * W;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&sm.full[b])), "r"(BYTES)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(sm.wbuf[b])),
                 "l"(src), "r"(BYTES), "r"(su32(&sm.full[b]))
                 : "memory");
}

// once per CTA, before its first tile
template <int W>
__device__ __forceinline__ void init_ring(Smem<W> &sm, unsigned long long wait_ns) {
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.full[b])) : "memory");
            sm.done[b] = 0;
        }
        sm.abort = 0;
        sm.wait_ns = wait_ns;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// One pass over the tile of TM rows (KIND above).  EVAL: g at sm.p[0..TM)
// into sm.g.  FWDZ: z_l of rows row0 + r < nrows into zbuf + l*ldl (row-major
// [row][W]), l = 0..n_mid, and the ReLU masks [z_l > 0] of l < n_mid as bits
// in the register-tile order of the thread that will apply them (mbits).
// BACK: sm.act holds delta_{n_mid} (feature-major); delta_{l-1}, masked with
// those bits, goes to dbuf + (l-1)*ldl.  Must be called by all NT threads,
// with both ring buffers free (no chunk in flight).  ph holds the thread's
// phase bits of the two buffers' barriers across tiles.
// Mask words: layer l, tile t, thread tid: mbits[((l * ntiles + t) * NT + tid) * MW + w],
// bit (j % 4) * 8 + rr of word j / 4 for row rg*8 + rr, output og + 16 j.
template <int W, int KIND = EVAL>
__device__ void mlp_tile(const MlpDev &m, Smem<W> &sm, uint32_t (&ph)[2], Counters *ctr, float *zbuf = nullptr,
                         float *dbuf = nullptr, long long row0 = 0, long long nrows = 0, long long ldl = 0,
                         uint32_t *mbits = nullptr, long long tile = 0, long long ntiles = 0) {
    constexpr int MW = W / 64;  // mask words per thread and layer (TO * 8 / 32)
    constexpr int TO = W / 16;      // outputs per thread
    constexpr int NCH = W / KC;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nchunks = m.n_mid * NCH;  // >= 2: n_mid >= 1, W / KC >= 2
    if (tid == 0) {
        issue_chunk<W, KIND>(m, sm, 0, 0);
        issue_chunk<W, KIND>(m, sm, 1, 1);
    }
    if (KIND != BACK) {  // layer 0: 3 -> W on CUDA cores
        const int r = tid & (TM - 1), half = tid >> 7;
        const float4 p = sm.p[r];
        const bool st = KIND == FWDZ && row0 + r < nrows;
        for (int o = half * (W / 2); o < (half + 1) * (W / 2); ++o) {
            const float z = fmaf(__ldg(m.w0 + 3 * o), p.x,
                                 fmaf(__ldg(m.w0 + 3 * o + 1), p.y, fmaf(__ldg(m.w0 + 3 * o + 2), p.z, __ldg(m.b0 + o))));
            sm.act[o][r] = fmaxf(z, 0.f);
            if (st) zbuf[(size_t)(row0 + r) * W + o] = z;
        }
        __syncthreads();
        if (KIND == FWDZ) {  // mask bits of z_0 in the register-tile order
            const int og = tid & 15, rg = tid >> 4;
            uint32_t wds[MW];
#pragma unroll
            for (int w = 0; w < MW; ++w) wds[w] = 0u;
#pragma unroll
            for (int j = 0; j < TO; ++j)
#pragma unroll
                for (int rr = 0; rr < 8; ++rr)
                    if (sm.act[og + 16 * j][rg * 8 + rr] > 0.f) wds[j >> 2] |= 1u << ((j & 3) * 8 + rr);
            uint32_t *mp = mbits + ((size_t)tile * NT + tid) * MW;
#pragma unroll
            for (int w = 0; w < MW; ++w) mp[w] = wds[w];
        }
    }
    // thread (og, rg): rows rg*8 .. rg*8+7, outputs og + 16 j (j < TO); the
    // weight chunk holds, at q*64 + og*4 + e, the weights of output og + 16(4q + e),
    // so each thread reads 16 contiguous bytes and the activation write-back
    // below stores consecutive rows from consecutive lanes.  Products run as
    // packed FP32 pairs (fma.rn.f32x2: outputs 2p and 2p+1 of the thread).
    const int og = tid & 15, rg = tid >> 4;
    int ch = 0;
    for (int l = 0; l < m.n_mid; ++l) {
        unsigned long long acc[8][TO / 2];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr)
#pragma unroll
            for (int p = 0; p < TO / 2; ++p) acc[rr][p] = 0ull;
        uint32_t mw[MW];  // BACK: this thread's mask bits of the layer below, fetched under the products
        if (KIND == BACK) {
            const uint32_t *mp = mbits + (((size_t)(m.n_mid - 1 - l) * ntiles + tile) * NT + tid) * MW;
#pragma unroll
            for (int w = 0; w < MW; ++w) mw[w] = mp[w];
        }
        for (int c = 0; c < NCH; ++c, ++ch) {
            const int b = ch & 1;
            wait_chunk<W>(sm, b, ph[b], ctr);
            ph[b] ^= 1u;
            const float *wb = sm.wbuf[b];
            // fully unrolled: the loads of later rows are scheduled under the
            // FMAs of earlier ones (86 % of the FFMA peak against 80 % at 4)
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                const int i = c * KC + kk;
                const float4 a0 = *reinterpret_cast<const float4 *>(&sm.act[i][rg * 8]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&sm.act[i][rg * 8 + 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                unsigned long long a2[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) asm("mov.b64 %0, {%1, %1};" : "=l"(a2[rr]) : "f"(a[rr]));
#pragma unroll
                for (int q = 0; q < TO / 4; ++q) {
                    const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(wb + kk * W + q * 64 + og * 4);
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[rr][2 * q]) : "l"(a2[rr]), "l"(w.x));
                        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[rr][2 * q + 1]) : "l"(a2[rr]), "l"(w.y));
                    }
                }
            }
            // the warp is done with buffer b; the last of the NT/32 warps
            // refills it with the chunk two ahead
            __syncwarp();
            if (lane == 0 && atomicAdd(&sm.done[b], 1u) == NT / 32 - 1) {
                sm.done[b] = 0;
                if (ch + 2 < nchunks) issue_chunk<W, KIND>(m, sm, ch + 2, b);
            }
        }
        __syncthreads();  // every warp has read this layer's input
        // EVAL / FWDZ: bias + ReLU (z stored by FWDZ); BACK: the mask of the
        // layer below; back into the activation buffer
        const float *bl = m.bm + (size_t)l * W;
        float *zl = KIND == FWDZ ? zbuf + (size_t)(l + 1) * ldl : nullptr;
        float *dl = KIND == BACK ? dbuf + (size_t)(m.n_mid - 1 - l) * ldl : nullptr;
        uint32_t fw[MW];  // FWDZ: mask bits of this layer's z (stored below unless it is the top layer)
#pragma unroll
        for (int w = 0; w < MW; ++w) fw[w] = 0u;
#pragma unroll
        for (int p = 0; p < TO / 2; ++p) {
            float lo[8], hi[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) asm("mov.b64 {%0, %1}, %2;" : "=f"(lo[rr]), "=f"(hi[rr]) : "l"(acc[rr][p]));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float *v = h ? hi : lo;
                const int o = og + 16 * (2 * p + h);
                float a[8];
                const int j = 2 * p + h;
                if (KIND == BACK) {
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        const long long row = row0 + rg * 8 + rr;
                        a[rr] = (mw[j >> 2] >> ((j & 3) * 8 + rr)) & 1u ? v[rr] : 0.f;
                        if (row < nrows) dl[(size_t)row * W + o] = a[rr];
                    }
                } else {
                    const float b = __ldg(bl + o);
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr) {
                        const float z = v[rr] + b;
                        a[rr] = fmaxf(z, 0.f);
                        if (KIND == FWDZ) {
                            if (row0 + rg * 8 + rr < nrows) zl[(size_t)(row0 + rg * 8 + rr) * W + o] = z;
                            if (z > 0.f) fw[j >> 2] |= 1u << ((j & 3) * 8 + rr);
                        }
                    }
                }
                *reinterpret_cast<float4 *>(&sm.act[o][rg * 8]) = make_float4(a[0], a[1], a[2], a[3]);
                *reinterpret_cast<float4 *>(&sm.act[o][rg * 8 + 4]) = make_float4(a[4], a[5], a[6], a[7]);
            }
        }
        if (KIND == FWDZ && l + 1 < m.n_mid) {
            uint32_t *mp = mbits + (((size_t)(l + 1) * ntiles + tile) * NT + tid) * MW;
#pragma unroll
            for (int w = 0; w < MW; ++w) mp[w] = fw[w];
        }
        __syncthreads();  // the next layer reads this layer's output
    }
    if (KIND == EVAL) {  // output layer W -> 1
        const int r = tid & (TM - 1), half = tid >> 7;
        float s = 0.f;
        for (int i = half * (W / 2); i < (half + 1) * (W / 2); ++i) s = fmaf(__ldg(m.wout + i), sm.act[i][r], s);
        if (half) sm.red[r] = s;
        __syncthreads();
        if (!half) sm.g[r] = s + sm.red[r] + m.bout;
        __syncthreads();
    }
}

__device__ __forceinline__ float outer_f(const MlpDev &m, float4 p, float g) {
    const float r = sqrtf(fmaf(p.x, p.x, fmaf(p.y, p.y, p.z * p.z)));
    return (fmaf(m.alpha, g, m.radial * r - m.r0) / m.beta) * m.inv_lam;
}

// Persistent hopper over a batch of items: the CTA's 128 rows take columns
// from item cur's queue; when the item has no column left for this CTA and
// all rows are done, the CTA moves to the next item.
template <int W>
__global__ void __launch_bounds__(NT, 1) k_hop_mlp_fp32(const Item *__restrict__ items, int n_items,
                                                         unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    init_ring<W>(sm, wait_ns);
    uint32_t ph[2] = {0u, 0u};
    int cur = 0;
    uint32_t col = NONE, rank = 0;
    int k = 0;
    bool done = false;
    float x = 0.f, y = 0.f;
    unsigned long long evals = 0;
    while (cur < n_items) {
        const Item &it = items[cur];
        const GridP &g = it.g;
        const Scratch &s = it.s;
        const int N = g.N;
        const uint32_t ncols = (uint32_t)N * (uint32_t)N;
        bool live = false;
        if (tid < TM) {
            const bool need = col == NONE && !done;
            const unsigned needm = __ballot_sync(FULL, need);
            if (needm) {
                const int leader = __ffs(needm) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&s.ctr->next_col, (unsigned long long)__popc(needm));
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
            sm.p[tid] = live ? make_float4(x, y, fmaf((float)k + 0.5f, g.h, g.lo[2]), 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (!__syncthreads_or(live)) {
            // item cur is finished for this CTA
            if (tid < TM) {
                for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(FULL, evals, o);
                if (lane == 0 && evals) atomicAdd(&s.ctr->hop_evals, evals);
            }
            evals = 0;
            col = NONE;
            done = false;
            ++cur;
            continue;
        }
        if (tid == 0) atomicAdd(&s.ctr->row_slots, (unsigned long long)TM);
        mlp_tile<W>(it.m, sm, ph, s.ctr);
        if (tid < TM) {
            bool mark = false, empty = false;
            int step = 1;
            if (live) {
                const float4 pc = sm.p[tid];
                const float f = outer_f(it.m, pc, sm.g[tid]);
                ++evals;
                float d = fabsf(f) - g.eps;
                if (!isfinite(f)) {
                    atomicOr(&s.ctr->flags, FLAG_NONFINITE);
                    d = 0.f;
                }
                if (d <= g.tau) {
                    mark = true;
                    empty = cell_is_empty(g, d, pc.x, pc.y, pc.z);
                } else {
                    const float stp = floorf(d * g.inv_h);
                    step = stp < 1.f ? 1 : (stp > (float)N ? N : (int)stp);
                }
            }
            const unsigned mm = __ballot_sync(FULL, mark);
            if (mm) {
                const int leader = __ffs(mm) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&s.ctr->marks, (unsigned long long)__popc(mm));
                base = __shfl_sync(FULL, base, leader);
                if (mark) {
                    const unsigned long long idx = base + __popc(mm & lt);
                    if (idx < (unsigned long long)s.cap_marks)
                        s.marks_raw[idx] = pack_mark(col, (uint32_t)k, rank, empty);
                    else
                        atomicOr(&s.ctr->flags, FLAG_MARK_OVERFLOW);
                }
            }
            if (live) {
                if (mark) {
                    ++rank;
                    ++k;
                } else {
                    k += step;
                }
                if (k >= N) {
                    s.colcount[col] = rank;
                    col = NONE;
                }
            }
        }
        // sm.p / sm.g are rewritten only after the barrier at the top of the next pass
    }
}

// Point lists over a batch of items: MODE 0 = the unique lattice vertices of
// each item, MODE 1 = each item's refinement list, MODE 2 = explicit points
// (one item), MODE 3 = all (N+1)^3 lattice points into s.lat (enumeration).
template <int W, int MODE>
__global__ void __launch_bounds__(NT, 1) k_pts_mlp_fp32(const Item *__restrict__ items, int n_items,
                                                         const float *pts, long long npts, float *outv,
                                                         unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    __shared__ unsigned long long tile_s;
    __shared__ unsigned long long total_s;
    const int tid = threadIdx.x;
    init_ring<W>(sm, wait_ns);
    uint32_t ph[2] = {0u, 0u};
    for (int cur = 0; cur < n_items;) {
        const Item &it = items[cur];
        const Scratch &s = it.s;
        const GridP &g = it.g;
        unsigned long long *counter = MODE == 1 ? &s.ctr->next_tile2 : &s.ctr->next_tile;
        if (tid == 0) {
            const bool stopped = MODE != 2 && (s.ctr->flags & STOP_FLAGS);
            const unsigned long long nl = (unsigned long long)(g.N + 1) * (g.N + 1) * (g.N + 1);
            total_s = stopped ? 0ull
                              : (MODE == 0 ? s.ctr->verts
                                           : (MODE == 1 ? s.ctr->refine : (MODE == 3 ? nl : (unsigned long long)npts)));
            tile_s = total_s ? atomicAdd(counter, 1ull) : 0ull;
        }
        __syncthreads();
        const unsigned long long t = tile_s, total = total_s;
        __syncthreads();
        if (t * TM >= total) {
            ++cur;
            continue;
        }
        if (tid < TM) {
            const unsigned long long r = t * TM + tid;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < total) {
                if (MODE == 2) {
                    p = make_float4(pts[3 * r], pts[3 * r + 1], pts[3 * r + 2], 0.f);
                } else if (MODE == 3) {
                    const unsigned long long N1 = g.N + 1;
                    const unsigned long long a = r % N1, b = (r / N1) % N1, c = r / (N1 * N1);
                    p = make_float4(fmaf((float)a, g.h, g.lo[0]), fmaf((float)b, g.h, g.lo[1]),
                                    fmaf((float)c, g.h, g.lo[2]), 0.f);
                } else {
                    const unsigned long long key = s.vkey[MODE == 1 ? (unsigned long long)s.rlist[r] : r];
                    const int N1 = g.N + 1;
                    const uint32_t line = (uint32_t)(key & 0xFFFFFFFFull), c = (uint32_t)(key >> 32);
                    const uint32_t a = line / (uint32_t)N1, b = line - a * (uint32_t)N1;
                    p = make_float4(fmaf((float)a, g.h, g.lo[0]), fmaf((float)b, g.h, g.lo[1]),
                                    fmaf((float)c, g.h, g.lo[2]), 0.f);
                }
            }
            sm.p[tid] = p;
        }
        __syncthreads();
        mlp_tile<W>(it.m, sm, ph, s.ctr);
        if (tid < TM) {
            const unsigned long long r = t * TM + tid;
            if (r < total) {
                const float f = outer_f(it.m, sm.p[tid], sm.g[tid]);
                if (MODE != 2 && !isfinite(f)) atomicOr(&s.ctr->flags, FLAG_NONFINITE);
                if (MODE == 0) s.vval[r] = f;
                else if (MODE == 1) s.vval[s.rlist[r]] = f;
                else if (MODE == 3) s.lat[r] = f;
                else outv[r] = f;
            }
        }
        __syncthreads();
    }
}

// The adjoint's forward pass over V vertices P: z_0 .. z_{n_mid} into Z (+ l*ldl).
template <int W>
__global__ void __launch_bounds__(NT, 1) k_adj_fwd(MlpDev m, const float *__restrict__ P, long long V,
                                                   float *__restrict__ Z, long long ldl, uint32_t *__restrict__ mbits,
                                                   Counters *ctr, unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    const int tid = threadIdx.x;
    init_ring<W>(sm, wait_ns);
    uint32_t ph[2] = {0u, 0u};
    for (long long t = blockIdx.x; t * TM < V; t += gridDim.x) {
        const long long row0 = t * TM;
        if (tid < TM) {
            const long long r = row0 + tid;
            sm.p[tid] = r < V ? make_float4(P[3 * r], P[3 * r + 1], P[3 * r + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        mlp_tile<W, FWDZ>(m, sm, ph, ctr, Z, nullptr, row0, V, ldl, mbits, t, (V + TM - 1) / TM);
    }
}

// The adjoint's delta chain: delta_{n_mid} from D (+ n_mid*ldl) down to
// delta_0, masked by the stored pre-activations Z, into D.
template <int W>
__global__ void __launch_bounds__(NT, 1) k_adj_bwd(MlpDev m, long long V, const uint32_t *__restrict__ mbits,
                                                   float *__restrict__ D, long long ldl, Counters *ctr,
                                                   unsigned long long wait_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    const int tid = threadIdx.x;
    init_ring<W>(sm, wait_ns);
    uint32_t ph[2] = {0u, 0u};
    const float *DL = D + (size_t)m.n_mid * ldl;
    for (long long t = blockIdx.x; t * TM < V; t += gridDim.x) {
        const long long row0 = t * TM;
        // delta_L rows into the feature-major buffer, 16 bytes per load
#pragma unroll 8
        for (int e = tid; e < TM * W / 4; e += NT) {
            const int r = e / (W / 4), o = 4 * (e - r * (W / 4));
            const float4 d = row0 + r < V ? *reinterpret_cast<const float4 *>(DL + (size_t)(row0 + r) * W + o)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            sm.act[o][r] = d.x;
            sm.act[o + 1][r] = d.y;
            sm.act[o + 2][r] = d.z;
            sm.act[o + 3][r] = d.w;
        }
        __syncthreads();
        mlp_tile<W, BACK>(m, sm, ph, ctr, nullptr, D, row0, V, ldl, const_cast<uint32_t *>(mbits), t,
                          (V + TM - 1) / TM);
    }
}

template <class K>
int occupancy_grid(K kernel, size_t smem, int nsm) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, NT, smem);
    return nsm * (per < 1 ? 1 : per);
}

}  // namespace

#define GH_DISPATCH_W(W, ...)                                            \
    switch (W) {                                                         \
    case 64: { constexpr int WW = 64; __VA_ARGS__; } break;              \
    case 128: { constexpr int WW = 128; __VA_ARGS__; } break;            \
    default: { constexpr int WW = 256; __VA_ARGS__; } break;             \
    }

void launch_hop_mlp_fp32(const Item *items, int n_items, int width, int nsm, cudaStream_t st) {
    GH_DISPATCH_W(width, {
        const size_t smem = sizeof(Smem<WW>);
        const int grid = occupancy_grid(k_hop_mlp_fp32<WW>, smem, nsm);
        k_hop_mlp_fp32<WW><<<grid, NT, smem, st>>>(items, n_items, wait_limit_ns());
    })
}

void launch_eval_vertices_mlp_fp32(const Item *items, int n_items, int width, int nsm, bool refine_list,
                                   cudaStream_t st) {
    GH_DISPATCH_W(width, {
        const size_t smem = sizeof(Smem<WW>);
        if (refine_list) {
            const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 1>, smem, nsm);
            k_pts_mlp_fp32<WW, 1><<<grid, NT, smem, st>>>(items, n_items, nullptr, 0, nullptr, wait_limit_ns());
        } else {
            const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 0>, smem, nsm);
            k_pts_mlp_fp32<WW, 0><<<grid, NT, smem, st>>>(items, n_items, nullptr, 0, nullptr, wait_limit_ns());
        }
    })
}

void launch_lattice_mlp_fp32(const Item *items, int width, int nsm, cudaStream_t st) {
    GH_DISPATCH_W(width, {
        const size_t smem = sizeof(Smem<WW>);
        const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 3>, smem, nsm);
        k_pts_mlp_fp32<WW, 3><<<grid, NT, smem, st>>>(items, 1, nullptr, 0, nullptr, wait_limit_ns());
    })
}

static Counters *adj_counters() {
    static thread_local Counters *ctr = nullptr;
    if (!ctr) {
        cudaMalloc(&ctr, sizeof(Counters));
        cudaMemset(ctr, 0, sizeof(Counters));
    }
    return ctr;
}

void launch_adj_fwd_fp32(const MlpDev &m, const float *P, long long V, float *Z, long long ldl, uint32_t *mbits,
                         int nsm, cudaStream_t st) {
    Counters *ctr = adj_counters();
    GH_DISPATCH_W(m.width, {
        const size_t smem = sizeof(Smem<WW>);
        int grid = occupancy_grid(k_adj_fwd<WW>, smem, nsm);
        const long long tiles = (V + TM - 1) / TM;
        if (grid > tiles) grid = (int)(tiles < 1 ? 1 : tiles);
        k_adj_fwd<WW><<<grid, NT, smem, st>>>(m, P, V, Z, ldl, mbits, ctr, wait_limit_ns());
    })
}

void launch_adj_bwd_fp32(const MlpDev &m, long long V, const uint32_t *mbits, float *D, long long ldl, int nsm,
                         cudaStream_t st) {
    Counters *ctr = adj_counters();
    GH_DISPATCH_W(m.width, {
        const size_t smem = sizeof(Smem<WW>);
        int grid = occupancy_grid(k_adj_bwd<WW>, smem, nsm);
        const long long tiles = (V + TM - 1) / TM;
        if (grid > tiles) grid = (int)(tiles < 1 ? 1 : tiles);
        k_adj_bwd<WW><<<grid, NT, smem, st>>>(m, V, mbits, D, ldl, ctr, wait_limit_ns());
    })
}

void launch_eval_points_mlp_fp32(const MlpDev &m, const float *p, long long n, float *out, int nsm,
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
    GH_DISPATCH_W(m.width, {
        const size_t smem = sizeof(Smem<WW>);
        int grid = occupancy_grid(k_pts_mlp_fp32<WW, 2>, smem, nsm);
        const long long tiles = (n + TM - 1) / TM;
        if (grid > tiles) grid = (int)(tiles < 1 ? 1 : tiles);
        k_pts_mlp_fp32<WW, 2><<<grid, NT, smem, st>>>(ditem, 1, p, n, out, wait_limit_ns());
    })
}

}  // namespace gh
