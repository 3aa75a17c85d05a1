// Derived layouts of a neural SDB's weights, built on the device from the
// packed parameter block W0[W][3] b0[W] { W_l[W][W] b_l[W] } x n_mid w_out[W]
// b_out, so that creating an SDB costs one upload and one launch.
//   wt  (FP32 evaluation engine): per layer [input i][output o], the outputs
//       of a row permuted so that position q*64 + og*4 + e holds output
//       og + 16(4q + e);
//   wtb (adjoint delta chain): per layer [output o][input i], the inputs
//       permuted the same way;
//   wbf (tensor-core engine): per layer, K-blocks of 64 inputs x W outputs in
//       the 128-byte swizzled K-major layout the MMA reads from shared memory
//       (row n, 16-byte chunk c of inputs [8c, 8c+8) at
//       (n/8)*1024 + (n%8)*128 + ((c ^ n%8) * 16)), BF16 rounded to nearest
//       even;
//   wx6 (split-BF16 engine): per layer three BF16 parts of every weight,
//       w = w_h + w_m + w_l exactly (w_h = bf16(w), w_m = bf16(w - w_h),
//       w_l = bf16(w - w_h - w_m)), stored part by part (low, middle, high),
//       each part in wbf's layout;
//   bm  hidden biases, n_mid x [W].
#include "gh_internal.cuh"

namespace gh {

namespace {

__device__ __forceinline__ int perm_pos(int o) {
    const int og = o & 15, m = o >> 4;
    return (m >> 2) * 64 + og * 4 + (m & 3);
}

// BF16 of an FP32 value, rounded to nearest even (finite values)
__device__ __forceinline__ uint16_t bf16_rne(float v) {
    const uint32_t u = __float_as_uint(v);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__global__ void __launch_bounds__(256) k_prep_mlp(const float *__restrict__ params, int W, int n_mid,
                                                  float *__restrict__ wt, float *__restrict__ wtb,
                                                  uint16_t *__restrict__ wbf, uint16_t *__restrict__ wx6,
                                                  float *__restrict__ bm) {
    const long long WW = (long long)W * W, total = (long long)n_mid * WW;
    const long long mid0 = 4LL * W;  // W0 and b0 come first
    const int KB = W / 64;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(e / WW);
        const long long r = e - l * WW;
        const int o = (int)(r / W), i = (int)(r - (long long)o * W);  // W_l[o][i]
        const float v = params[mid0 + l * (WW + W) + r];
        wt[l * WW + (long long)i * W + perm_pos(o)] = v;
        wtb[l * WW + (long long)o * W + perm_pos(i)] = v;
        const int kb = i >> 6, kk = i & 63;
        const int byte = (o >> 3) * 1024 + (o & 7) * 128 + (((kk >> 3) ^ (o & 7)) << 4) + (kk & 7) * 2;
        const uint16_t hi = bf16_rne(v);
        wbf[((long long)l * KB + kb) * W * 64 + byte / 2] = hi;
        const float rem = v - bf16_val(hi);  // exact
        const uint16_t mid = bf16_rne(rem);
        const uint16_t low = bf16_rne(rem - bf16_val(mid));
        const uint16_t parts[3] = {low, mid, hi};
        for (int p = 0; p < 3; ++p)
            wx6[(((long long)l * 3 + p) * KB + kb) * W * 64 + byte / 2] = parts[p];
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n_mid * W;
         e += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(e / W), o = (int)(e - (long long)l * W);
        bm[e] = params[mid0 + l * (WW + W) + WW + o];
    }
}

}  // namespace

void launch_prep_mlp(const float *params, int W, int n_mid, float *wt, float *wtb, uint16_t *wbf, uint16_t *wx6,
                     float *bm, cudaStream_t st) {
    k_prep_mlp<<<1024, 256, 0, st>>>(params, W, n_mid, wt, wtb, wbf, wx6, bm);
}

}  // namespace gh
