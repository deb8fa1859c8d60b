// Kernel instantiations for 3-D elements in double (see fr_kernels.cuh).
#include "fr_kernels.cuh"

namespace frk {

cudaError_t launch_3_f64(int N, int kind, bool visc, const KArgs<double> &a, int grid, cudaStream_t s) {
    switch (N) {
    case 1: return launch_n<3, 1, double>(kind, visc, a, grid, s);
    case 2: return launch_n<3, 2, double>(kind, visc, a, grid, s);
    case 3: return launch_n<3, 3, double>(kind, visc, a, grid, s);
    case 4: return launch_n<3, 4, double>(kind, visc, a, grid, s);
    case 5: return launch_n<3, 5, double>(kind, visc, a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
static cudaError_t prepare_n(bool visc) {
    cudaError_t e;
    if (visc) e = prep_smem(k_flux<3, N, double, true>, smem_bytes<3, N, double>(K_FLUX, true));
    else e = prep_smem(k_flux<3, N, double, false>, smem_bytes<3, N, double>(K_FLUX, false));
    if (e != cudaSuccess) return e;
    // adaptive steps (their own instantiations, register level 0)
    if (visc) e = prep_smem(k_flux<3, N, double, true, 0, true>, smem_bytes<3, N, double>(K_FLUX, true));
    else e = prep_smem(k_flux<3, N, double, false, 0, true>, smem_bytes<3, N, double>(K_FLUX, false));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_grad<3, N, double>, smem_bytes<3, N, double>(K_GRAD, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_interp<3, N, double>, smem_bytes<3, N, double>(K_INTERP, false));
    if (e != cudaSuccess || !visc) return e;
    e = prep_smem(k_stage<3, N, double>, smem_bytes<3, N, double>(K_STAGE, true));
    if (e != cudaSuccess) return e;
    e = prep_smem(k_stage<3, N, double, 0, true>, smem_bytes<3, N, double>(K_STAGE, true));
    if (e != cudaSuccess) return e;
    return prep_smem(k_interp_visc<3, N, double>, smem_bytes<3, N, double>(K_INTERP_VISC, true));
}

cudaError_t prepare_3_f64(int N, bool visc) {
    switch (N) {
    case 1: return prepare_n<1>(visc);
    case 2: return prepare_n<2>(visc);
    case 3: return prepare_n<3>(visc);
    case 4: return prepare_n<4>(visc);
    case 5: return prepare_n<5>(visc);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t mortar_3_f64(const MArgs<double> &a, cudaStream_t s) {
    return launch_mortar<3, double>(a, s);
}

}  // namespace frk
