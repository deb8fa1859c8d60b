// Kernel instantiations for 2-D elements in float (see fr_kernels.cuh).
#include "fr_kernels.cuh"

namespace frk {

cudaError_t launch_2_f32(int N, int kind, bool visc, const KArgs<float> &a, int grid, cudaStream_t s) {
    switch (N) {
    case 1: return launch_n<2, 1, float>(kind, visc, a, grid, s);
    case 2: return launch_n<2, 2, float>(kind, visc, a, grid, s);
    case 3: return launch_n<2, 3, float>(kind, visc, a, grid, s);
    case 4: return launch_n<2, 4, float>(kind, visc, a, grid, s);
    case 5: return launch_n<2, 5, float>(kind, visc, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
static cudaError_t prepare_n(bool visc) {
    cudaError_t e;
    if (visc) e = prep_smem(k_flux<2, N, float, true>, smem_bytes<2, N, float>(K_FLUX, true));
    else e = prep_smem(k_flux<2, N, float, false>, smem_bytes<2, N, float>(K_FLUX, false));
    if (e != cudaSuccess) return e;
    // adaptive steps (their own instantiations, register level 0)
    if (visc) e = prep_smem(k_flux<2, N, float, true, 0, true>, smem_bytes<2, N, float>(K_FLUX, true));
    else e = prep_smem(k_flux<2, N, float, false, 0, true>, smem_bytes<2, N, float>(K_FLUX, false));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_grad<2, N, float>, smem_bytes<2, N, float>(K_GRAD, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_interp<2, N, float>, smem_bytes<2, N, float>(K_INTERP, false));
    if (e != cudaSuccess || !visc) return e;
    e = prep_smem(k_stage<2, N, float>, smem_bytes<2, N, float>(K_STAGE, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_stage<2, N, float, 0, true>, smem_bytes<2, N, float>(K_STAGE, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_interp_visc<2, N, float>, smem_bytes<2, N, float>(K_INTERP_VISC, true));
    if (e != cudaSuccess || !has_level1<N, float>()) return e;
    // register level 1 (autotuner candidates)
    constexpr int L1 = has_level1<N, float>() ? 1 : 0;
    e = prep_smem(k_flux<2, N, float, true, L1>, smem_bytes<2, N, float>(K_FLUX, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_grad<2, N, float, L1>, smem_bytes<2, N, float>(K_GRAD, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_stage<2, N, float, L1>, smem_bytes<2, N, float>(K_STAGE, true));
    if (e != cudaSuccess) return e;
    constexpr int L2 = has_level1<N, float>() ? 2 : 0;
    e = prep_smem(k_flux<2, N, float, true, L2>, smem_bytes<2, N, float>(K_FLUX, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_grad<2, N, float, L2>, smem_bytes<2, N, float>(K_GRAD, true));
    if (e != cudaSuccess) return e;
    return prep_smem(k_stage<2, N, float, L2>, smem_bytes<2, N, float>(K_STAGE, true));
}

cudaError_t prepare_2_f32(int N, bool visc) {
    switch (N) {
    case 1: return prepare_n<1>(visc);
    case 2: return prepare_n<2>(visc);
    case 3: return prepare_n<3>(visc);
    case 4: return prepare_n<4>(visc);
    case 5: return prepare_n<5>(visc);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t mortar_2_f32(const MArgs<float> &a, cudaStream_t s) {
    return launch_mortar<2, float>(a, s);
}

}  // namespace frk
