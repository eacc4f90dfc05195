// ICD sweep kernels with __nv_bfloat16 stored matrix values (one translation unit
// per value type, so the library's device code compiles in parallel).
#include "sweep.cuh"

sweep_fn mace_sweep_kernel_bf16(int max_views, int K, bool nb26, bool det)
{
    return sweep_lookup<__nv_bfloat16>(max_views, K, nb26, det);
}

sweep_queue_fn mace_sweep_queue_kernel_bf16(int max_views, bool nb26, int W, int K)
{
    return sweep_queue_lookup<__nv_bfloat16>(max_views, nb26, W, K);
}
