// lbch_pair.cu -- launch and set-up of the two-step kernel (periodic instances, tau_g = 1), f32 and f64.
#include "lbch_internal.h"
#include "lbch_pair.cuh"

namespace lbch {
namespace {

template <typename C, typename P, int TX, int TY, int NT>
cudaError_t launch_pair_v(lbch_handle* h, int parity)
{
    using L = PairShape<C, P, TX, TY>;
    const lbch_handle::PerShape& ps = h->pr[h->pshape];
    PairArgs<C, P> a;
    a.inst0 = h->inst[0];
    a.inst = h->d_inst;
    a.tile_begin = ps.d_tile_begin;
    a.ttabs = static_cast<const C*>(ps.d_ttabs);
    static_assert(L::TAB_STRIDE * sizeof(C) == L::TAB_BYTES, "the host lays the tables out with this stride");
    a.n_inst = h->n_inst;
    a.total_tiles = ps.total_tiles;
    a.pitch = h->pitch;
    a.phi_in = static_cast<const P*>(h->phi[parity]);
    a.lo_in = h->lo[parity];
    a.phi_out = static_cast<P*>(h->phi[parity ^ 1]);
    a.lo_out = h->lo[parity ^ 1];
    a.ctl = h->ctl;
    a.t_off = h->t_off;
    a.t_adv = h->t_adv;
    a.need_time = h->need_time;
    a.debug_skip = h->debug_skip;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ps.grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = L::BYTES;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->no_pdl ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return h->n_inst == 1 ? cudaLaunchKernelEx(&cfg, ch_pair_kernel<C, P, TX, TY, NT, true>, a)
                          : cudaLaunchKernelEx(&cfg, ch_pair_kernel<C, P, TX, TY, NT, false>, a);
}

template <typename C, typename P, int TX, int TY, int NT>
cudaError_t prepare_pair_v(lbch_handle* h, int k)
{
    using L = PairShape<C, P, TX, TY>;
    const void* kern = reinterpret_cast<const void*>(ch_pair_kernel<C, P, TX, TY, NT, false>);
    cudaError_t e = lbch_kernel_smem(kern, h->device, L::BYTES);
    if (e == cudaSuccess)
        e = lbch_kernel_smem(reinterpret_cast<const void*>(ch_pair_kernel<C, P, TX, TY, NT, true>), h->device, L::BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = lbch_kernel_fit(kern, h->device, NT, L::BYTES, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    h->pr[k].grid = std::max(1, std::min(h->pr[k].total_tiles, per_sm * sms));
    return cudaSuccess;
}

}  // namespace
}  // namespace lbch

// The shapes are those of pair_shape() (lbch_internal.h), in its order.
cudaError_t lbch_launch_pair(lbch_handle* h, int parity)
{
    using namespace lbch;
    const int k = h->pshape;
    if (k < 0 || k >= kPairShapes || !h->pr[k].d_tile_begin || h->pr[k].grid < 1) return cudaErrorInvalidValue;
    if (h->prec == LBCH_F64)
        return k == 0 ? launch_pair_v<double, double, 32, 8, 512>(h, parity)
             : k == 1 ? launch_pair_v<double, double, 16, 8, 256>(h, parity)
             : k == 2 ? launch_pair_v<double, double, 16, 16, 512>(h, parity) : launch_pair_v<double, double, 32, 14, 1024>(h, parity);
    return k == 0 ? launch_pair_v<float, float, 32, 16, 768>(h, parity)
         : k == 1 ? launch_pair_v<float, float, 32, 14, 1024>(h, parity)
         : k == 2 ? launch_pair_v<float, float, 32, 16, 1024>(h, parity) : launch_pair_v<float, float, 32, 8, 512>(h, parity);
}

cudaError_t lbch_prepare_pair(lbch_handle* h, int k)
{
    using namespace lbch;
    if (h->prec == LBCH_F64)
        return k == 0 ? prepare_pair_v<double, double, 32, 8, 512>(h, k)
             : k == 1 ? prepare_pair_v<double, double, 16, 8, 256>(h, k)
             : k == 2 ? prepare_pair_v<double, double, 16, 16, 512>(h, k) : prepare_pair_v<double, double, 32, 14, 1024>(h, k);
    return k == 0 ? prepare_pair_v<float, float, 32, 16, 768>(h, k)
         : k == 1 ? prepare_pair_v<float, float, 32, 14, 1024>(h, k)
         : k == 2 ? prepare_pair_v<float, float, 32, 16, 1024>(h, k) : prepare_pair_v<float, float, 32, 8, 512>(h, k);
}
