// lbch_sweep_launch.cuh -- launch and set-up of the row-sweep kernel for one precision; included by the
// per-precision translation units, so that their kernels compile in parallel.
#pragma once
#include "lbch_internal.h"
#include "lbch_sweep.cuh"

namespace lbch {

template <typename C, typename S, typename P, bool FF, int TY, int NW, bool GEN, bool COMPACT, bool M3>
cudaError_t launch_sweep_v(lbch_handle* h, int parity)
{
    using L = SweepShape<P, S, FF, TY, NW, GEN>;
    const lbch_handle::PerShape& ps = h->sw[h->shape];
    SweepArgs<C, S, P> a;
    a.inst0 = h->inst[0];
    a.inst = h->d_inst;
    a.tile_begin = ps.d_tile_begin;
    a.tiles = ps.d_tiles;
    a.tabs = tables<C>(h);
    a.n_inst = h->n_inst;
    a.total_tiles = ps.total_tiles;
    a.pitch = h->pitch;
    a.debug_skip = h->debug_skip;
    a.phi_out = static_cast<P*>(h->phi[parity ^ 1]);
    a.lo_out = h->lo[parity ^ 1];
    a.ctl = h->ctl;
    a.t_off = h->t_off;
    a.t_adv = h->t_adv;
    a.need_time = h->need_time;
    a.g_out = static_cast<S*>(h->g[parity ^ 1]);
    a.rows = h->rows;
    a.H_in = M3 ? static_cast<const C*>(h->H[parity]) : nullptr;
    a.H_out = M3 ? static_cast<C*>(h->H[parity ^ 1]) : nullptr;
    a.H_plane = (long long)h->rows * h->pitch;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(GEN ? ps.grid_gen : ps.grid);
    cfg.blockDim = dim3(NW * 32);
    cfg.dynamicSmemBytes = L::BYTES;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->no_pdl ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a single instance's record is read from the launch parameters (ch_sweep_kernel's SINGLE form)
    if (h->n_inst == 1)
        return cudaLaunchKernelEx(&cfg, ch_sweep_kernel<C, S, P, FF, TY, NW, GEN, COMPACT, true, M3>,
                                  ps.tm_phi[parity], ps.tm_lo[parity], h->tm_grow[parity], h->tm_lorow[parity], a);
    return cudaLaunchKernelEx(&cfg, ch_sweep_kernel<C, S, P, FF, TY, NW, GEN, COMPACT, false, M3>, ps.tm_phi[parity],
                              ps.tm_lo[parity], h->tm_grow[parity], h->tm_lorow[parity], a);
}

template <typename C, typename S, typename P, bool FF, int TY, int NW, bool COMPACT, bool M3>
cudaError_t launch_sweep_g(lbch_handle* h, int parity)
{
    return sweep_gen(h) ? launch_sweep_v<C, S, P, FF, TY, NW, true, COMPACT, M3>(h, parity)
                        : launch_sweep_v<C, S, P, FF, TY, NW, false, COMPACT, M3>(h, parity);
}

// M3 (Model III handles) is built for the two unrolled configurations only (kM3SweepShapes).
template <typename C, typename S, typename P, bool FF, bool M3>
cudaError_t launch_sweep_t(lbch_handle* h, int parity)
{
    if constexpr (M3) {
        switch (h->shape) {
        case 0: return launch_sweep_g<C, S, P, FF, 12, 4, false, true>(h, parity);
        case 1: return launch_sweep_g<C, S, P, FF, 6, 4, false, true>(h, parity);
        default: return cudaErrorInvalidValue;
        }
    } else {
        switch (h->shape) {
        case 0: return launch_sweep_g<C, S, P, FF, 12, 4, false, false>(h, parity);
        case 1: return launch_sweep_g<C, S, P, FF, 6, 4, false, false>(h, parity);
        case 2: return launch_sweep_g<C, S, P, FF, 6, 2, true, false>(h, parity);
        default: return launch_sweep_g<C, S, P, FF, 3, 4, true, false>(h, parity);
        }
    }
}

// Dynamic shared memory of one sweep kernel and the persistent grid that fits the device.
template <typename C, typename S, typename P, bool FF, int TY, int NW, bool GEN, bool COMPACT, bool M3>
cudaError_t prepare_sweep_v(lbch_handle* h, int k)
{
    using L = SweepShape<P, S, FF, TY, NW, GEN>;
    const void* kern = reinterpret_cast<const void*>(ch_sweep_kernel<C, S, P, FF, TY, NW, GEN, COMPACT, false, M3>);
    cudaError_t e = lbch_kernel_smem(kern, h->device, L::BYTES);
    if (e == cudaSuccess)
        e = lbch_kernel_smem(reinterpret_cast<const void*>(ch_sweep_kernel<C, S, P, FF, TY, NW, GEN, COMPACT, true, M3>),
                             h->device, L::BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = lbch_kernel_fit(kern, h->device, NW * 32, L::BYTES, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    (GEN ? h->sw[k].grid_gen : h->sw[k].grid) = std::max(1, std::min(h->sw[k].total_tiles, per_sm * sms));
    return cudaSuccess;
}

template <typename C, typename S, typename P, bool FF, int TY, int NW, bool COMPACT, bool M3>
cudaError_t prepare_sweep_g(lbch_handle* h, int k)
{
    cudaError_t e = prepare_sweep_v<C, S, P, FF, TY, NW, true, COMPACT, M3>(h, k);
    if (e == cudaSuccess && h->tau1) e = prepare_sweep_v<C, S, P, FF, TY, NW, false, COMPACT, M3>(h, k);
    return e;
}

template <typename C, typename S, typename P, bool FF, bool M3>
cudaError_t prepare_sweep_t(lbch_handle* h, int k)
{
    if constexpr (M3) {
        return k == 0 ? prepare_sweep_g<C, S, P, FF, 12, 4, false, true>(h, k)
             : k == 1 ? prepare_sweep_g<C, S, P, FF, 6, 4, false, true>(h, k) : cudaErrorInvalidValue;
    } else {
        return k == 0 ? prepare_sweep_g<C, S, P, FF, 12, 4, false, false>(h, k)
             : k == 1 ? prepare_sweep_g<C, S, P, FF, 6, 4, false, false>(h, k)
             : k == 2 ? prepare_sweep_g<C, S, P, FF, 6, 2, true, false>(h, k)
                      : prepare_sweep_g<C, S, P, FF, 3, 4, true, false>(h, k);
    }
}

}  // namespace lbch
