// lbch_sweep_f32.cu -- the row-sweep step kernels of the f32 path.
#include "lbch_sweep_launch.cuh"

cudaError_t lbch_launch_sweep_f32(lbch_handle* h, int parity)
{
    return lbch::launch_sweep_t<float, float, float, true, false>(h, parity);
}

cudaError_t lbch_prepare_sweep_f32(lbch_handle* h, int k)
{
    return lbch::prepare_sweep_t<float, float, float, true, false>(h, k);
}
