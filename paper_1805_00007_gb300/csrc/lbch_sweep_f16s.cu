// lbch_sweep_f16s.cu -- the row-sweep step kernels of the f16s path.
#include "lbch_sweep_launch.cuh"

cudaError_t lbch_launch_sweep_f16s(lbch_handle* h, int parity)
{
    return lbch::launch_sweep_t<float, __half, float, false, false>(h, parity);
}

cudaError_t lbch_prepare_sweep_f16s(lbch_handle* h, int k)
{
    return lbch::prepare_sweep_t<float, __half, float, false, false>(h, k);
}
