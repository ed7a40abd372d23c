// lbch_sweep_f16s_m3.cu -- the row-sweep step kernels of the f16s path for handles with a Model III
// instance (Eq. F2-1 in full), in a translation unit of their own so that they compile in parallel.
#include "lbch_sweep_launch.cuh"

cudaError_t lbch_launch_sweep_f16s_m3(lbch_handle* h, int parity)
{
    return lbch::launch_sweep_t<float, __half, float, false, true>(h, parity);
}

cudaError_t lbch_prepare_sweep_f16s_m3(lbch_handle* h, int k)
{
    return lbch::prepare_sweep_t<float, __half, float, false, true>(h, k);
}
