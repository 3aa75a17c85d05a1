// Neural SDB in BF16 on the tcgen05 tensor cores (placeholder until the
// tensor-core kernels land; bf16_supported() reports false).
#include "gh_internal.cuh"

namespace gh {
bool bf16_supported(int) { return false; }
void launch_hop_mlp_bf16(const MlpDev &, const GridP &, Scratch &, int, cudaStream_t) {}
void launch_eval_vertices_mlp_bf16(const MlpDev &, const GridP &, Scratch &, int, cudaStream_t) {}
void launch_eval_points_mlp_bf16(const MlpDev &, const float *, long long, float *, int, cudaStream_t) {}
void launch_refine_select(const GridP &, Scratch &, cudaStream_t) {}
}  // namespace gh
