// Implicit-surface adjoint of a neural SDB (gh_backward).
//
// A mesh vertex v that stays on the level set f(v; theta) = 0 moves with the
// parameters as dv/dtheta = -grad_x f (df/dtheta) / |grad_x f|^2, so a loss on
// the vertices has
//   dL/dtheta = sum_v s_v df/dtheta(v),  s_v = -(dL/dv . grad_x f(v)) / |grad_x f(v)|^2.
// For f = (rad |p| - r0 + alpha g(p)) / (beta lambda) (rad = 0 for a network
// given without the radial term) and g a ReLU MLP
//   z_0 = W_0 p + b_0, z_l = W_l relu(z_{l-1}) + b_l (l = 1..L), g = w . relu(z_L) + b,
// back-propagation gives delta_L = w * [z_L > 0], delta_{l-1} = (W_l^T delta_l) *
// [z_{l-1} > 0], dg/dp = W_0^T delta_0, and with c = alpha / (beta lambda)
//   dL/dW_l = c sum_v s_v delta_l relu(z_{l-1})^T,  dL/db_l = c sum_v s_v delta_l,
//   dL/dW_0 = c sum_v s_v delta_0 p^T,  dL/dw = c sum_v s_v relu(z_L),  dL/db = c sum_v s_v.
// The activations are recomputed from the vertices (nothing is kept from the
// polygonization).  Over a chunk of vertices the forward pass (storing every
// z_l) and the delta chain run on the FP32 tile engine of the network's
// evaluation (k_mlp_fp32.cu); the weight sums are dense FP32 products on the
// FFMA pipe (k_gemm, 128 x 128 tiles, 8 x 8 per thread in packed FP32 pairs,
// register-prefetched 16-deep K slices); the
// sums over vertices use a split over the vertex axis whose partial results
// are added in a fixed order, so the gradient is deterministic.
#include <math.h>
#include <string.h>

#include <vector>

#include "gh_internal.cuh"

namespace gh {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, GT = 256, PADS = 4;

// C[M x N] (+ split z: C + z*M*ldc) = sum_k opA(m,k) opB(k,n) over the k-range
// [z*kchunk, (z+1)*kchunk) with opA(m,k) = (TA ? A[k*lda+m] : A[m*lda+k]),
// relu'd if RA and scaled by ksc[k]; opB likewise.  Epilogue: + bias[n],
// then * [mask[m*ldc+n] > 0].
// 128 x 128 tile per CTA, 8 x 8 per thread as packed FP32 pairs
// (fma.rn.f32x2); the next 16-deep K slice is fetched into registers while
// the current one is multiplied out of the other shared-memory buffer.
template <bool TA, bool TB, bool RA, bool RB>
__global__ void __launch_bounds__(GT) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                             const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                             const float *__restrict__ bias, const float *__restrict__ mask,
                                             const float *__restrict__ ksc, int kchunk) {
    __shared__ __align__(16) float As[2][BK][BM + PADS];
    __shared__ __align__(16) float Bs[2][BK][BN + PADS];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    // each thread stages 8 elements of A and 8 of B per slice: element
    // e = tid + 256 r (r < 8) of the 128 x 16 slice, walking the contiguous
    // direction of the operand's storage fastest
    float ra[8], rb[8];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = tid + r * GT;  // 0..2047
            {
                const int mm = TA ? (e & (BM - 1)) : (e >> 4), kk = TA ? (e >> 7) : (e & (BK - 1));
                const int m = m0 + mm, k = k0 + kk;
                float v = 0.f;
                if (m < M && k < ke) {
                    v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
                    if (RA) v = fmaxf(v, 0.f);
                    if (ksc) v *= ksc[k];
                }
                ra[r] = v;
            }
            {
                const int nn = TB ? (e >> 4) : (e & (BN - 1)), kk = TB ? (e & (BK - 1)) : (e >> 7);
                const int n = n0 + nn, k = k0 + kk;
                float v = 0.f;
                if (n < N && k < ke) {
                    v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
                    if (RB) v = fmaxf(v, 0.f);
                }
                rb[r] = v;
            }
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = tid + r * GT;
            const int mm = TA ? (e & (BM - 1)) : (e >> 4), ka = TA ? (e >> 7) : (e & (BK - 1));
            const int nn = TB ? (e >> 4) : (e & (BN - 1)), kbb = TB ? (e & (BK - 1)) : (e >> 7);
            As[buf][ka][mm] = ra[r];
            Bs[buf][kbb][nn] = rb[r];
        }
    };
    unsigned long long acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0ull;
    int buf = 0;
    if (kb < ke) {
        fetch(kb);
        stash(0);
    }
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += BK) {
        const bool more = k0 + BK < ke;
        if (more) fetch(k0 + BK);  // in flight during the products below
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8 + 4]);
            const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(&Bs[buf][kk][tx * 8]);
            const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(&Bs[buf][kk][tx * 8 + 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const unsigned long long b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                unsigned long long a2;
                asm("mov.b64 %0, {%1, %1};" : "=l"(a2) : "f"(a[i]));
#pragma unroll
                for (int j = 0; j < 4; ++j) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[i][j]) : "l"(a2), "l"(b[j]));
            }
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    float *Cz = C + (size_t)blockIdx.z * M * ldc;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty * 8 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[i][j]));
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int n = n0 + tx * 8 + 2 * j + u;
                if (n >= N) continue;
                float v = u ? hi : lo;
                if (bias) v += bias[n];
                if (mask && !(mask[(size_t)m * ldc + n] > 0.f)) v = 0.f;
                Cz[(size_t)m * ldc + n] = v;
            }
        }
    }
}

template <bool TA, bool TB, bool RA, bool RB>
void gemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc, const float *bias,
          const float *mask, const float *ksc, int splits, cudaStream_t st) {
    const int kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    k_gemm<TA, TB, RA, RB><<<grid, GT, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ksc, kchunk);
}

// delta_L = w * [z_L > 0]
__global__ void k_adj_top(const float *__restrict__ ZL, int V, const float *__restrict__ wout, int W,
                          float *__restrict__ D) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)V * W;
         e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e % W);
        D[e] = ZL[e] > 0.f ? wout[o] : 0.f;
    }
}

// grad_x f from delta_0, then s_v
__global__ void k_adj_s(const float *__restrict__ P, const float *__restrict__ dL, int V,
                        const float *__restrict__ D0, const float *__restrict__ w0, int W, float alpha, float inv_bl,
                        float radial, float *__restrict__ s) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v < V; v += nw) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int o = lane; o < W; o += 32) {
            const float d = D0[(size_t)v * W + o];
            gx = fmaf(w0[3 * o], d, gx);
            gy = fmaf(w0[3 * o + 1], d, gy);
            gz = fmaf(w0[3 * o + 2], d, gz);
        }
        for (int off = 16; off > 0; off >>= 1) {
            gx += __shfl_xor_sync(0xFFFFFFFFu, gx, off);
            gy += __shfl_xor_sync(0xFFFFFFFFu, gy, off);
            gz += __shfl_xor_sync(0xFFFFFFFFu, gz, off);
        }
        if (lane == 0) {
            const float px = P[3 * v], py = P[3 * v + 1], pz = P[3 * v + 2];
            const float r = sqrtf(px * px + py * py + pz * pz);
            const float ir = r > 0.f ? radial / r : 0.f;
            const float fx = (px * ir + alpha * gx) * inv_bl;
            const float fy = (py * ir + alpha * gy) * inv_bl;
            const float fz = (pz * ir + alpha * gz) * inv_bl;
            const float n2 = fx * fx + fy * fy + fz * fz;
            const float dot = dL[3 * v] * fx + dL[3 * v + 1] * fy + dL[3 * v + 2] * fz;
            s[v] = n2 > 0.f ? -dot / n2 : 0.f;
        }
    }
}

// out[i] (+)= c * sum_z part[z][i], z in increasing order
__global__ void k_adj_reduce(const float *__restrict__ part, int splits, long long n, float c, float *__restrict__ out,
                             int accumulate) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < splits; ++z) acc += part[(size_t)z * n + i];
        out[i] = accumulate ? __fadd_rn(out[i], __fmul_rn(c, acc)) : __fmul_rn(c, acc);
    }
}

// part[z][j * NP + a] = sum over rows v of split z of s[v] * X'[v][j] *
// P[v][a] (NP = 3) or s[v] * X'[v][j] (NP = 1), with X' = relu(X) if RELU,
// X' = 1 if X is null.  Column sums of the parameter gradients that have one
// (or three) outputs per unit: b_l, W_0, w_out.  A block of 32 columns x 8
// row groups: group g adds the split's rows v = g, g + 8, ... in order, and
// the 8 group sums are added in group order -- a fixed summation order.
template <int NP, bool RELU>
__global__ void __launch_bounds__(256) k_colsum(const float *__restrict__ X, int V, int W, const float *__restrict__ s,
                                                const float *__restrict__ P, int rows_per_split,
                                                float *__restrict__ part) {
    __shared__ float red[8][32][NP];
    const int z = blockIdx.y, cx = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + cx;
    const int v0 = z * rows_per_split, v1 = min(V, v0 + rows_per_split);
    float acc[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) acc[a] = 0.f;
    if (j < W) {
#pragma unroll 4
        for (int v = v0 + g; v < v1; v += 8) {
            float x = X ? X[(size_t)v * W + j] : 1.f;
            if (RELU) x = fmaxf(x, 0.f);
            const float sx = s[v] * x;
            if (NP == 1) {
                acc[0] += sx;
            } else {
#pragma unroll
                for (int a = 0; a < NP; ++a) acc[a] = fmaf(sx, P[3 * v + a], acc[a]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < NP; ++a) red[g][cx][a] = acc[a];
    __syncthreads();
    if (g == 0 && j < W) {
#pragma unroll
        for (int a = 0; a < NP; ++a) {
            float t = red[0][cx][a];
            for (int q = 1; q < 8; ++q) t += red[q][cx][a];
            part[(size_t)z * W * NP + (size_t)j * NP + a] = t;
        }
    }
}

template <int NP, bool RELU>
void colsum(const float *X, int V, int W, const float *s, const float *P, int splits, float *part, cudaStream_t st) {
    const int rows = (V + splits - 1) / splits;
    dim3 grid((W + 31) / 32, splits);
    k_colsum<NP, RELU><<<grid, 256, 0, st>>>(X, V, W, s, P, rows, part);
}

__global__ void k_fill(float *p, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

size_t adjoint_buffer_floats(int W, int n_mid, int VC, int splits) {
    const size_t L1 = (size_t)n_mid + 1;
    const size_t mask_words = (size_t)n_mid * ((VC + 127) / 128) * 256 * (W / 64);
    return L1 * VC * W * 2 + VC + (size_t)splits * W * W + VC + mask_words;
}

// One chunk of vertices; accumulates into grad (packed like the parameters).
void adjoint_chunk(const MlpDev &m, const float *P, const float *dL, int V, float *grad, bool accumulate,
                   const AdjBuffers &b, cudaStream_t st) {
    const int W = m.width, L = m.n_mid, S = b.splits;
    const float c = m.alpha / m.beta * m.inv_lam;
    float *Zl[17], *Dl[17];
    for (int l = 0; l <= L; ++l) {
        Zl[l] = b.Z + (size_t)l * b.VC * W;
        Dl[l] = b.D + (size_t)l * b.VC * W;
    }
    const int eb = 1024;
    // forward: pre-activations of every layer; backward chain of g (both on the
    // FP32 tile engine of the network's evaluation)
    const long long ldl = (long long)b.VC * W;
    launch_adj_fwd_fp32(m, P, V, b.Z, ldl, b.mbits, b.nsm, st);
    k_adj_top<<<eb, 256, 0, st>>>(Zl[L], V, m.wout, W, Dl[L]);
    launch_adj_bwd_fp32(m, V, b.mbits, b.D, ldl, b.nsm, st);
    k_adj_s<<<(V + 7) / 8, 256, 0, st>>>(P, dL, V, Dl[0], m.w0, W, m.alpha, 1.f / m.beta * m.inv_lam, m.radial, b.s);
    // parameter gradients: sums over the vertices of the chunk
    const size_t oW0 = 0, ob0 = (size_t)3 * W, omid = ob0 + W;
    const size_t ow = omid + (size_t)L * ((size_t)W * W + W);
    const int gb = 512;
    // W_0 and b_0
    colsum<3, false>(Dl[0], V, W, b.s, P, S, b.part, st);
    k_adj_reduce<<<gb, 256, 0, st>>>(b.part, S, (long long)W * 3, c, grad + oW0, accumulate);
    colsum<1, false>(Dl[0], V, W, b.s, nullptr, S, b.part, st);
    k_adj_reduce<<<gb, 256, 0, st>>>(b.part, S, (long long)W, c, grad + ob0, accumulate);
    for (int l = 1; l <= L; ++l) {
        const size_t oW = omid + (size_t)(l - 1) * ((size_t)W * W + W), ob = oW + (size_t)W * W;
        gemm<true, false, false, true>(W, W, V, Dl[l], W, Zl[l - 1], W, b.part, W, nullptr, nullptr, b.s, S, st);
        k_adj_reduce<<<gb, 256, 0, st>>>(b.part, S, (long long)W * W, c, grad + oW, accumulate);
        colsum<1, false>(Dl[l], V, W, b.s, nullptr, S, b.part, st);
        k_adj_reduce<<<gb, 256, 0, st>>>(b.part, S, (long long)W, c, grad + ob, accumulate);
    }
    // output layer: w_out from relu(z_L), b_out from the scales alone
    colsum<1, true>(Zl[L], V, W, b.s, nullptr, S, b.part, st);
    k_adj_reduce<<<gb, 256, 0, st>>>(b.part, S, (long long)W, c, grad + ow, accumulate);
    colsum<1, false>(nullptr, V, 1, b.s, nullptr, S, b.part, st);
    k_adj_reduce<<<1, 32, 0, st>>>(b.part, S, 1, c, grad + ow + W, accumulate);
}

void adjoint_fill_ones(float *p, long long n, cudaStream_t st) { k_fill<<<256, 256, 0, st>>>(p, n, 1.f); }

// ---------------------------------------------------------------------------
// Adjoint of an analytic (CSG) SDB.  The min / max fold selects one
// primitive a at each vertex (the running value is replaced only by a
// strictly smaller union term or a strictly larger subtract / intersect
// term), so f = sgn d_a with sgn = -1 for a subtracted primitive.  With
// q = Rot (v - c):
//   sphere  d = |q| - r                  dd/dq = q/|q|,  dd/dr = -1
//   torus   a = |(qx,qz)| - R, d = |(a,qy)| - r
//           dd/dq = (a qx/|(qx,qz)|, qy, a qz/|(qx,qz)|) / |(a,qy)|, dd/dR = -a/|(a,qy)|, dd/dr = -1
//   box     e = |q| - h; outside: d = |max(e,0)|, dd/dq = sign(q) max(e,0)/d, dd/dh = -max(e,0)/d;
//           inside: d = max_k e_k, dd/dq_k = sign(q_k), dd/dh_k = -1 (largest k)
//   capsule d = |q - (0, clamp(qy,-H,H), 0)| - r; the clamp moves with H past the caps
//   cylinder, hexagonal prism: the box rule in 2-D on (e0, |qy| - H), e0 the
//           radial (resp. folded hexagon) distance, differentiated through the
//           fold's mirror
//   cone    distance to the nearer of the base segment and the slant segment in
//           (rho, qy); the closest point's derivative in R and H is that of its
//           segment's parametrisation (base: (min(rho,R), -H); slant: (R - tR, 2tH - H))
//   prism and cone take the outward normal of the nearest edge or segment as the
//   direction wherever the closest point is inside it: at a mesh vertex p lies
//   on the surface and p - closest is rounding noise
// dd/dv = Rot^T dd/dq and dd/dc = -dd/dv.  Each vertex contributes
// s_v df/dtheta_a to its primitive a only.
// ---------------------------------------------------------------------------
__device__ float csg_prim_grad(const Prim &P, float x, float y, float z, float *gv, float *gs) {
    const float dx = x - P.c[0], dy = y - P.c[1], dz = z - P.c[2];
    const float *R = P.rot;
    const float q0 = R[0] * dx + R[1] * dy + R[2] * dz;
    const float q1 = R[3] * dx + R[4] * dy + R[5] * dz;
    const float q2 = R[6] * dx + R[7] * dy + R[8] * dz;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, val;
    gs[0] = gs[1] = gs[2] = 0.f;
    if (P.type == GH_PRIM_SPHERE) {
        const float n = sqrtf(q0 * q0 + q1 * q1 + q2 * q2);
        val = n - P.p[0];
        if (n > 0.f) {
            g0 = q0 / n;
            g1 = q1 / n;
            g2 = q2 / n;
        }
        gs[0] = -1.f;
    } else if (P.type == GH_PRIM_TORUS) {
        const float rxz = sqrtf(q0 * q0 + q2 * q2);
        const float a = rxz - P.p[0];
        const float n = sqrtf(a * a + q1 * q1);
        val = n - P.p[1];
        if (n > 0.f) {
            g0 = rxz > 0.f ? a * q0 / (rxz * n) : 0.f;
            g1 = q1 / n;
            g2 = rxz > 0.f ? a * q2 / (rxz * n) : 0.f;
            gs[0] = -a / n;
        }
        gs[1] = -1.f;
    } else if (P.type == GH_PRIM_CAPSULE) {
        // u = q - (0, clamp(qy, -H, H), 0), d = |u| - r
        const float H = P.p[0];
        const float yc = fminf(fmaxf(q1, -H), H), u1 = q1 - yc;
        const float n = sqrtf(q0 * q0 + u1 * u1 + q2 * q2);
        val = n - P.p[1];
        if (n > 0.f) {
            g0 = q0 / n;
            g1 = u1 / n;
            g2 = q2 / n;
            gs[0] = q1 > H ? -u1 / n : (q1 < -H ? u1 / n : 0.f);
        }
        gs[1] = -1.f;
    } else if (P.type == GH_PRIM_CYLINDER || P.type == GH_PRIM_HEXPRISM) {
        // e0: radial (cylinder) or hexagon (prism) distance, e1 = |qy| - H
        float e0, d0x = 0.f, d0z = 0.f, d0p = -1.f;
        if (P.type == GH_PRIM_CYLINDER) {
            const float rho = sqrtf(q0 * q0 + q2 * q2);
            e0 = rho - P.p[0];
            if (rho > 0.f) {
                d0x = q0 / rho;
                d0z = q2 / rho;
            }
        } else {
            // folded hexagon: |x|, |z|, then the mirror at 30 degrees
            const float a = P.p[0];
            const float sx = q0 < 0.f ? -1.f : 1.f, sz = q2 < 0.f ? -1.f : 1.f;
            float x = fabsf(q0), z = fabsf(q2);
            const float mx = -0.5f, mz = 0.8660254037844386f;
            const float dot = x * mx + z * mz;
            const bool refl = dot > 0.f;
            if (refl) {
                x -= 2.f * dot * mx;
                z -= 2.f * dot * mz;
            }
            const float lim = a * 0.5773502691896258f;
            const float v0 = x - a, v1 = z - fminf(fmaxf(z, -lim), lim);
            const float n = sqrtf(v0 * v0 + v1 * v1), sg = v0 < 0.f ? -1.f : 1.f;
            e0 = sg * n;
            float gx = 1.f, gz = 0.f;  // inside the edge's span: its outward normal
            d0p = -1.f;
            if (v1 != 0.f && n > 0.f) {  // past a corner: the corner's direction
                gx = sg * v0 / n;
                gz = sg * v1 / n;
                const float dv1 = z > lim ? -0.5773502691896258f : 0.5773502691896258f;
                d0p = sg * (-v0 + v1 * dv1) / n;
            }
            if (refl) {  // the mirror is its own transpose
                const float gd = gx * mx + gz * mz;
                gx -= 2.f * gd * mx;
                gz -= 2.f * gd * mz;
            }
            d0x = sx * gx;
            d0z = sz * gz;
        }
        const float e1 = fabsf(q1) - P.p[1];
        float w0, w1;
        if (e0 > 0.f || e1 > 0.f) {
            const float o0 = fmaxf(e0, 0.f), o1 = fmaxf(e1, 0.f), n = sqrtf(o0 * o0 + o1 * o1);
            val = n;
            w0 = o0 / n;
            w1 = o1 / n;
        } else {
            val = fmaxf(e0, e1);
            w0 = e0 >= e1 ? 1.f : 0.f;
            w1 = e0 >= e1 ? 0.f : 1.f;
        }
        g0 = w0 * d0x;
        g2 = w0 * d0z;
        g1 = w1 * (q1 < 0.f ? -1.f : 1.f);
        gs[0] = w0 * d0p;
        gs[1] = -w1;
    } else if (P.type == GH_PRIM_CONE) {
        const float R = P.p[0], H = P.p[1];
        const float rho = sqrtf(q0 * q0 + q2 * q2), y = q1;
        const float bs = fminf(fmaxf(rho, 0.f), R);
        const float b0 = rho - bs, b1 = y + H, db = sqrtf(b0 * b0 + b1 * b1);
        const float e0 = -R, e1 = 2.f * H;
        float t = ((rho - R) * e0 + (y + H) * e1) / (e0 * e0 + e1 * e1);
        t = fminf(fmaxf(t, 0.f), 1.f);
        const float s0 = rho - (R + t * e0), s1 = y - (-H + t * e1), ds = sqrtf(s0 * s0 + s1 * s1);
        const bool inside = y > -H && y < H && rho * 2.f * H < R * (H - y);
        const float sg = inside ? -1.f : 1.f;
        // gradient direction: the segment's outward normal where the closest
        // point lies inside the segment (at a surface point p - closest is
        // rounding noise), the direction from the closest end point otherwise
        float nr, ny, cR0, cH1, n;
        if (db < ds) {
            n = db;
            cR0 = rho > R ? 1.f : 0.f;  // d(closest)/dR = (cR0, 0), d(closest)/dH = (0, cH1)
            cH1 = -1.f;
            nr = 0.f;
            ny = -1.f;
            if (rho > R) {
                nr = n > 0.f ? sg * b0 / n : 0.f;
                ny = n > 0.f ? sg * b1 / n : 0.f;
            }
        } else {
            n = ds;
            cR0 = 1.f - t;
            cH1 = 2.f * t - 1.f;
            const float il = rsqrtf(e0 * e0 + e1 * e1);
            nr = e1 * il;
            ny = -e0 * il;
            if (t <= 0.f || t >= 1.f) {
                nr = n > 0.f ? sg * s0 / n : 0.f;
                ny = n > 0.f ? sg * s1 / n : 0.f;
            }
        }
        val = sg * n;
        if (rho > 0.f) {
            g0 = nr * q0 / rho;
            g2 = nr * q2 / rho;
        }
        g1 = ny;
        gs[0] = -nr * cR0;
        gs[1] = -ny * cH1;
    } else {
        const float q[3] = {q0, q1, q2};
        float e[3], o2 = 0.f, g[3] = {0.f, 0.f, 0.f};
        int km = 0;
        for (int k = 0; k < 3; ++k) {
            e[k] = fabsf(q[k]) - P.p[k];
            if (e[k] > 0.f) o2 += e[k] * e[k];
            if (e[k] > e[km]) km = k;
        }
        if (o2 > 0.f) {
            const float n = sqrtf(o2);
            val = n;
            for (int k = 0; k < 3; ++k) {
                const float mk = e[k] > 0.f ? e[k] / n : 0.f;
                g[k] = q[k] < 0.f ? -mk : mk;
                gs[k] = -mk;
            }
        } else {
            val = e[km];
            g[km] = q[km] < 0.f ? -1.f : 1.f;
            gs[km] = -1.f;
        }
        g0 = g[0];
        g1 = g[1];
        g2 = g[2];
    }
    gv[0] = R[0] * g0 + R[3] * g1 + R[6] * g2;
    gv[1] = R[1] * g0 + R[4] * g1 + R[7] * g2;
    gv[2] = R[2] * g0 + R[5] * g1 + R[8] * g2;
    return val;
}

__device__ float csg_prim_val(const Prim &P, float x, float y, float z) {
    float gv[3], gs[3];
    return csg_prim_grad(P, x, y, z, gv, gs);
}

__global__ void k_csg_adj_vertex(const Prim *__restrict__ prims, int nprim, const float *__restrict__ V,
                                 const float *__restrict__ dL, int nv, int *__restrict__ act,
                                 float *__restrict__ contrib) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const float x = V[3 * v], y = V[3 * v + 1], z = V[3 * v + 2];
        int a = 0;
        float sgn = 1.f, f = csg_prim_val(prims[0], x, y, z);
        for (int n = 1; n < nprim; ++n) {
            const float d = csg_prim_val(prims[n], x, y, z);
            const int op = prims[n].op;
            if (op == GH_OP_UNION) {
                if (d < f) { f = d; a = n; sgn = 1.f; }
            } else if (op == GH_OP_SUBTRACT) {
                if (-d > f) { f = -d; a = n; sgn = -1.f; }
            } else {
                if (d > f) { f = d; a = n; sgn = 1.f; }
            }
        }
        float gv[3], gs[3];
        csg_prim_grad(prims[a], x, y, z, gv, gs);
        const float gx = sgn * gv[0], gy = sgn * gv[1], gz = sgn * gv[2];
        const float g2 = gx * gx + gy * gy + gz * gz;
        const float sv = g2 > 0.f ? -(dL[3 * v] * gx + dL[3 * v + 1] * gy + dL[3 * v + 2] * gz) / g2 : 0.f;
        act[v] = a;
        float *o = contrib + (size_t)6 * v;
        o[0] = -sv * gx;
        o[1] = -sv * gy;
        o[2] = -sv * gz;
        o[3] = sv * sgn * gs[0];
        o[4] = sv * sgn * gs[1];
        o[5] = sv * sgn * gs[2];
    }
}

// one block per primitive: fixed-order sums over the vertices it was active at
__global__ void __launch_bounds__(256) k_csg_adj_reduce(const int *__restrict__ act, const float *__restrict__ contrib,
                                                         int nv, float *__restrict__ out) {
    __shared__ float red[6][256];
    const int prim = blockIdx.x;
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int v = threadIdx.x; v < nv; v += blockDim.x)
        if (act[v] == prim)
            for (int k = 0; k < 6; ++k) acc[k] += contrib[(size_t)6 * v + k];
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 20) {
        float val = 0.f;
        if (threadIdx.x >= 2 && threadIdx.x < 8) val = red[threadIdx.x - 2][0];
        out[(size_t)20 * prim + threadIdx.x] = val;
    }
}

void csg_adjoint(const Prim *prims, int nprim, const float *V, const float *dL, int nv, int *act, float *contrib,
                 float *out, cudaStream_t st) {
    if (nv > 0) k_csg_adj_vertex<<<(nv + 255) / 256 < 4096 ? (nv + 255) / 256 : 4096, 256, 0, st>>>(
        prims, nprim, V, dL, nv, act, contrib);
    k_csg_adj_reduce<<<nprim, 256, 0, st>>>(act, contrib, nv, out);
}

}  // namespace gh
