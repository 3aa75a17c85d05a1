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
    int abort;                   // a chunk wait timed out: stop waiting
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

// waits for the phase of the given parity of buffer b's barrier; after 2 s
// sets the abort bit (later waits return at once) and the timeout flag
template <int W>
__device__ __noinline__ void wait_chunk(Smem<W> &sm, int b, uint32_t parity, Counters *ctr) {
    if (mbar_try(&sm.full[b], parity)) return;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(&sm.full[b], parity)) return;
        if (*(volatile int *)&sm.abort) return;
        if ((it & 255) == 0 && gtimer() - t0 > WAIT_NS) {
            atomicOr((int *)&sm.abort, 1);
            atomicOr(&ctr->flags, FLAG_TIMEOUT);
            return;
        }
    }
}

// chunk ch of the hidden layers (K rows ch*KC.. of layer ch/NCH) into buffer b
template <int W>
__device__ __forceinline__ void issue_chunk(const MlpDev &m, Smem<W> &sm, int ch, int b) {
    constexpr int NCH = W / KC;
    constexpr uint32_t BYTES = KC * W * 4;
    const int l = ch / NCH, c = ch - l * NCH;
    const float *src = m.wt + (size_t)l * W * W + (size_t)c * KC * W;
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
__device__ __forceinline__ void init_ring(Smem<W> &sm) {
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.full[b])) : "memory");
            sm.done[b] = 0;
        }
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Evaluates g at sm.p[0..TM) into sm.g.  Must be called by all NT threads,
// with both ring buffers free (no chunk in flight).  ph holds the thread's
// phase bits of the two buffers' barriers across tiles.
template <int W>
__device__ void mlp_tile(const MlpDev &m, Smem<W> &sm, uint32_t (&ph)[2], Counters *ctr) {
    constexpr int TO = W / 16;      // outputs per thread
    constexpr int NCH = W / KC;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nchunks = m.n_mid * NCH;  // >= 2: n_mid >= 1, W / KC >= 2
    if (tid == 0) {
        issue_chunk<W>(m, sm, 0, 0);
        issue_chunk<W>(m, sm, 1, 1);
    }
    {  // layer 0: 3 -> W on CUDA cores
        const int r = tid & (TM - 1), half = tid >> 7;
        const float4 p = sm.p[r];
        for (int o = half * (W / 2); o < (half + 1) * (W / 2); ++o) {
            const float z = fmaf(__ldg(m.w0 + 3 * o), p.x,
                                 fmaf(__ldg(m.w0 + 3 * o + 1), p.y, fmaf(__ldg(m.w0 + 3 * o + 2), p.z, __ldg(m.b0 + o))));
            sm.act[o][r] = fmaxf(z, 0.f);
        }
    }
    __syncthreads();
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
                if (ch + 2 < nchunks) issue_chunk<W>(m, sm, ch + 2, b);
            }
        }
        __syncthreads();  // every warp has read this layer's input
        // bias + ReLU, back into the activation buffer
        const float *bl = m.bm + (size_t)l * W;
#pragma unroll
        for (int p = 0; p < TO / 2; ++p) {
            float lo[8], hi[8];
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) asm("mov.b64 {%0, %1}, %2;" : "=f"(lo[rr]), "=f"(hi[rr]) : "l"(acc[rr][p]));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float *v = h ? hi : lo;
                const int o = og + 16 * (2 * p + h);
                const float b = __ldg(bl + o);
                float4 v0, v1;
                v0.x = fmaxf(v[0] + b, 0.f);
                v0.y = fmaxf(v[1] + b, 0.f);
                v0.z = fmaxf(v[2] + b, 0.f);
                v0.w = fmaxf(v[3] + b, 0.f);
                v1.x = fmaxf(v[4] + b, 0.f);
                v1.y = fmaxf(v[5] + b, 0.f);
                v1.z = fmaxf(v[6] + b, 0.f);
                v1.w = fmaxf(v[7] + b, 0.f);
                *reinterpret_cast<float4 *>(&sm.act[o][rg * 8]) = v0;
                *reinterpret_cast<float4 *>(&sm.act[o][rg * 8 + 4]) = v1;
            }
        }
        __syncthreads();  // the next layer reads this layer's output
    }
    {  // output layer W -> 1
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
__global__ void __launch_bounds__(NT, 1) k_hop_mlp_fp32(const Item *__restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    init_ring<W>(sm);
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
                        col = (uint32_t)c;
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
            bool mark = false;
            int step = 1;
            if (live) {
                const float f = outer_f(it.m, sm.p[tid], sm.g[tid]);
                ++evals;
                float d = fabsf(f) - g.eps;
                if (!isfinite(f)) {
                    atomicOr(&s.ctr->flags, FLAG_NONFINITE);
                    d = 0.f;
                }
                if (d <= g.tau) {
                    mark = true;
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
                        s.marks_raw[idx] = pack_mark(col, (uint32_t)k, rank);
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
                                                         const float *pts, long long npts, float *outv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<W> &sm = *reinterpret_cast<Smem<W> *>(smem_raw);
    __shared__ unsigned long long tile_s;
    __shared__ unsigned long long total_s;
    const int tid = threadIdx.x;
    init_ring<W>(sm);
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
        k_hop_mlp_fp32<WW><<<grid, NT, smem, st>>>(items, n_items);
    })
}

void launch_eval_vertices_mlp_fp32(const Item *items, int n_items, int width, int nsm, bool refine_list,
                                   cudaStream_t st) {
    GH_DISPATCH_W(width, {
        const size_t smem = sizeof(Smem<WW>);
        if (refine_list) {
            const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 1>, smem, nsm);
            k_pts_mlp_fp32<WW, 1><<<grid, NT, smem, st>>>(items, n_items, nullptr, 0, nullptr);
        } else {
            const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 0>, smem, nsm);
            k_pts_mlp_fp32<WW, 0><<<grid, NT, smem, st>>>(items, n_items, nullptr, 0, nullptr);
        }
    })
}

void launch_lattice_mlp_fp32(const Item *items, int width, int nsm, cudaStream_t st) {
    GH_DISPATCH_W(width, {
        const size_t smem = sizeof(Smem<WW>);
        const int grid = occupancy_grid(k_pts_mlp_fp32<WW, 3>, smem, nsm);
        k_pts_mlp_fp32<WW, 3><<<grid, NT, smem, st>>>(items, 1, nullptr, 0, nullptr);
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
        k_pts_mlp_fp32<WW, 2><<<grid, NT, smem, st>>>(ditem, 1, p, n, out);
    })
}

}  // namespace gh
