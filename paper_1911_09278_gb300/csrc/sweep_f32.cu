// ICD sweep kernels with float stored matrix values (one translation unit
// per value type, so the library's device code compiles in parallel).
#include "sweep.cuh"

sweep_fn mace_sweep_kernel_f32(int max_views, int K, bool nb26, bool det)
{
    return sweep_lookup<float>(max_views, K, nb26, det);
}

sweep_queue_fn mace_sweep_queue_kernel_f32(int max_views, bool nb26, int W, int K)
{
    return sweep_queue_lookup<float>(max_views, nb26, W, K);
}
