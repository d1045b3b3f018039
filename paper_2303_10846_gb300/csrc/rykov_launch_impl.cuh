// Definitions of the launch sequences (included by kern_f64.cu / kern_f32.cu only).
#pragma once

#include "rykov_dev_packed.cuh"
#include "rykov_launch.cuh"

namespace rk {

constexpr int FACE_BS = 256;
constexpr int FACE_WPB = 8;         // faces (warps) per block of the interior-face kernel
constexpr int MICRO_WPB = 8;        // cells (warps) per block of the micro sweep
constexpr int RECON_WPB = 8;        // cells (warps) per block of the reconstruction

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

template <typename T>
cudaError_t Launch<T>::setup(const Dev<T>& d, cudaStream_t s) {
    k_setup_dt<T><<<d.N, 128, 0, s>>>(d);
    k_setup_lsq<T><<<cdiv(d.N, 128), 128, 0, s>>>(d);
    k_setup_face<T><<<cdiv(d.F, 256), 256, 0, s>>>(d);
    k_setup_slotT<T><<<cdiv(d.nnz > d.F ? d.nnz : d.F, 256), 256, 0, s>>>(d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::set_state(const Dev<T>& d, cudaStream_t s, const double* prim,
                                 const double* q) {
    k_set_state<T><<<d.N, 128, 0, s>>>(d, prim, q);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::recon(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    k_iter_begin<T><<<1, 1, 0, s>>>(d);
    pf.begin(0, s);
    if constexpr (std::is_same<T, float>::value) {
        if (d.packed)
            k_recon_p<RECON_WPB><<<cdiv(d.N, RECON_WPB), RECON_WPB * 32, 0, s>>>(d);
        else
            k_recon<T, RECON_WPB><<<cdiv(d.N, RECON_WPB), RECON_WPB * 32, 0, s>>>(d);
    } else {
        k_recon<T, RECON_WPB><<<cdiv(d.N, RECON_WPB), RECON_WPB * 32, 0, s>>>(d);
    }
    pf.end(s);
    pf.launches += 2;
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::faces_interior(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    if (d.Fi) {
        pf.begin(1, s);
        constexpr int FW = sizeof(T) == 4 ? FACE_FW : 1;
        k_face_interior<T, FACE_WPB, FW><<<cdiv(d.Fi, FACE_WPB / FW), FACE_WPB * 32, 0, s>>>(d);
        pf.end(s);
        pf.launches += 1;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::faces_boundary(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    if (d.Fb) {
        pf.begin(2, s);
        k_face_boundary<T, FACE_BS><<<d.Fb, FACE_BS, 0, s>>>(d);
        pf.end(s);
        pf.launches += 1;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::faces(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    cudaError_t e = faces_interior(d, s, pf);
    return e != cudaSuccess ? e : faces_boundary(d, s, pf);
}

template <typename T>
cudaError_t Launch<T>::fluxes(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    pf.begin(3, s);
    k_face_radius<T><<<cdiv(d.F, 256), 256, 0, s>>>(d);
    k_cell_macro_flux<T><<<cdiv(d.N, 256), 256, 0, s>>>(d);
    pf.end(s);
    pf.launches += 2;
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::micro_flux(const Dev<T>& d, cudaStream_t s, Prof& pf) {
    pf.begin(3, s);
    k_micro_flux<T, MICRO_WPB><<<cdiv(d.N, MICRO_WPB), MICRO_WPB * 32, 0, s>>>(d);
    pf.end(s);
    pf.launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::macro(const Dev<T>& d, cudaStream_t s, const Sched& sc, int n_macro,
                             Prof& pf) {
    pf.begin(4, s);
    const int C = (int)sc.col_off.size() - 1;
    if (sc.macro32) {
        // FP32 delta form (mixed contexts): per-colour launches, each overlapping the
        // launch of the next (programmatic stream serialisation) unless sc.pdl is 0
        k_macro_prep32<T><<<cdiv(d.N, 128), 128, 0, s>>>(d);
        pf.launches += 1;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        for (int it = 0; it < n_macro; ++it) {
            for (int dir = 0; dir < 2; ++dir) {
                for (int cc = 0; cc < C; ++cc) {
                    const int col = dir == 0 ? cc : C - 1 - cc;
                    const int lo = sc.col_off[col], n = sc.col_off[col + 1] - lo;
                    if (!n) continue;
                    const int ln = sc.macro_lanes;
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3((unsigned)cdiv((long long)n * ln, 128));
                    cfg.blockDim = dim3(128);
                    cfg.stream = s;
                    cfg.attrs = attr;
                    cfg.numAttrs = sc.pdl ? 1 : 0;
                    const int ff = (int)(it == 0 && dir == 0);
                    const cudaError_t e =
                        ln == 1 ? cudaLaunchKernelEx(&cfg, k_macro_sweep32<T, 1>, d, lo, n, col, ff)
                        : ln == 4 ? cudaLaunchKernelEx(&cfg, k_macro_sweep32<T, 4>, d, lo, n, col, ff)
                                  : cudaLaunchKernelEx(&cfg, k_macro_sweep32<T, 2>, d, lo, n, col, ff);
                    if (e != cudaSuccess) return e;
                    pf.launches += 1;
                }
            }
        }
        k_macro_finish<T><<<cdiv(d.N, 128), 128, 0, s>>>(d, 1);
        pf.end(s);
        pf.launches += 1;
        return cudaGetLastError();
    }
    k_macro_prep<T><<<cdiv(d.N, 128), 128, 0, s>>>(d);
    pf.launches += 1;
    bool done = false;
    if (sc.coop_grid > 0 && n_macro > 0) {
        // all sweeps in one cooperative launch (grid barriers between colours)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(sc.coop_grid);
        cfg.blockDim = dim3(128);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_macro_coop<T>, d, sc.col_cell, d.col_off_d, C, n_macro, d.bar,
                                           sc.coop_extra, sc.coop_limit_ns);
        if (e == cudaSuccess) {
            pf.launches += 1;
            done = true;
        } else {
            (void)cudaGetLastError();
        }
    }
    // per-colour phases, each overlapping the launch of the next (programmatic stream
    // serialisation) unless sc.pdl is 0
    cudaLaunchAttribute pattr[1];
    pattr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pattr[0].val.programmaticStreamSerializationAllowed = 1;
    for (int it = 0; it < n_macro && !done; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int cc = 0; cc < C; ++cc) {
                const int col = dir == 0 ? cc : C - 1 - cc;
                const int lo = sc.col_off[col], n = sc.col_off[col + 1] - lo;
                if (!n) continue;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)cdiv((long long)n * MACRO_LANES, 128));
                cfg.blockDim = dim3(128);
                cfg.stream = s;
                cfg.attrs = pattr;
                cfg.numAttrs = sc.pdl ? 1 : 0;
                const cudaError_t e = cudaLaunchKernelEx(&cfg, k_macro_sweep<T>, d, (const int*)sc.col_cell, lo, n, col,
                                                         (int)(it == 0 && dir == 0));
                if (e != cudaSuccess) return e;
                pf.launches += 1;
            }
        }
    }
    k_macro_finish<T><<<cdiv(d.N, 128), 128, 0, s>>>(d, 0);
    pf.end(s);
    pf.launches += 1;
    return cudaGetLastError();
}

// dynamic shared memory of one block of the staged micro sweep
template <typename T>
struct StBytes {
    template <bool FIRST, bool LAST>
    static size_t get(int maxs) {
        return (size_t)MICRO_ST_WPB * 2 * (2 * maxs + 4) * 32 * micro_nv<T, FIRST, LAST>() * sizeof(T);
    }
};

template <typename T>
cudaError_t Launch<T>::micro(const Dev<T>& d, cudaStream_t s, const Sched& sc, int n_micro,
                             Prof& pf) {
    const int C = (int)sc.col_off.size() - 1;
    const int nsw = 2 * n_micro;
    for (int sw = 0; sw < nsw; ++sw) {
        const int dir = sw & 1;
        for (int cc = 0; cc < C; ++cc) {
            const int col = dir == 0 ? cc : C - 1 - cc;
            const int lo = sc.col_off[col], n = sc.col_off[col + 1] - lo;
            if (!n) continue;
            // the first sweep forms Res for every cell of this colour; the last
            // sweep applies the update and the Step-6 sums
            pf.begin(sw == 0 ? 5 : (sw == nsw - 1 ? 7 : 6), s);
            const int* cl = sc.col_cell + lo;
            const int kind = sw == 0 ? 0 : (sw == nsw - 1 ? 2 : 1);
            bool done = false;
            if constexpr (std::is_same<T, float>::value) {
                if (d.packed && ((sc.staged >> kind) & 1)) {
                    constexpr int W = MICRO_ST_WPB;
                    const dim3 g(cdiv(n, W)), b(W * 32);
                    const int mx = sc.maxs;
                    const size_t sb = sw == 0 ? StBytes<T>::template get<true, false>(mx)
                                              : (sw == nsw - 1 ? StBytes<T>::template get<false, true>(mx)
                                                               : StBytes<T>::template get<false, false>(mx));
                    if ((sc.staged >> 3) & 1) {            // the cell's own rows by bulk copies
                        if (sw == 0) k_micro_sweep_st_p<W, true, false, true><<<g, b, sb, s>>>(d, cl, n, col, mx);
                        else if (sw == nsw - 1) k_micro_sweep_st_p<W, false, true, true><<<g, b, sb, s>>>(d, cl, n, col, mx);
                        else k_micro_sweep_st_p<W, false, false, true><<<g, b, sb, s>>>(d, cl, n, col, mx);
                    } else {
                        if (sw == 0) k_micro_sweep_st_p<W, true, false, false><<<g, b, sb, s>>>(d, cl, n, col, mx);
                        else if (sw == nsw - 1) k_micro_sweep_st_p<W, false, true, false><<<g, b, sb, s>>>(d, cl, n, col, mx);
                        else k_micro_sweep_st_p<W, false, false, false><<<g, b, sb, s>>>(d, cl, n, col, mx);
                    }
                    done = true;
                } else if (d.packed) {
                    const dim3 g(cdiv(n, MICRO_WPB)), b(MICRO_WPB * 32);
                    if (sw == 0) k_micro_sweep_p<MICRO_WPB, true, false><<<g, b, 0, s>>>(d, cl, n, col);
                    else if (sw == nsw - 1) k_micro_sweep_p<MICRO_WPB, false, true><<<g, b, 0, s>>>(d, cl, n, col);
                    else k_micro_sweep_p<MICRO_WPB, false, false><<<g, b, 0, s>>>(d, cl, n, col);
                    done = true;
                }
            }
            if (done) {
            } else if ((sc.staged >> kind) & 1) {
                constexpr int W = MICRO_ST_WPB;
                const dim3 g(cdiv(n, W)), b(W * 32);
                const int mx = sc.maxs;
                if (sw == 0)
                    k_micro_sweep_st<T, W, true, false><<<g, b, StBytes<T>::template get<true, false>(mx), s>>>(d, cl, n, col, mx);
                else if (sw == nsw - 1)
                    k_micro_sweep_st<T, W, false, true><<<g, b, StBytes<T>::template get<false, true>(mx), s>>>(d, cl, n, col, mx);
                else
                    k_micro_sweep_st<T, W, false, false><<<g, b, StBytes<T>::template get<false, false>(mx), s>>>(d, cl, n, col, mx);
            } else {
                const dim3 g(cdiv(n, MICRO_WPB)), b(MICRO_WPB * 32);
                if (sw == 0) k_micro_sweep<T, MICRO_WPB, true, false><<<g, b, 0, s>>>(d, cl, n, col);
                else if (sw == nsw - 1) k_micro_sweep<T, MICRO_WPB, false, true><<<g, b, 0, s>>>(d, cl, n, col);
                else k_micro_sweep<T, MICRO_WPB, false, false><<<g, b, 0, s>>>(d, cl, n, col);
            }
            pf.end(s);
            pf.launches += 1;
        }
    }
    pf.begin(8, s);
    k_cell_update<T><<<cdiv(d.N, 128), 128, 0, s>>>(d);
    k_residual_reduce<T><<<1, 256, 0, s>>>(d, cdiv(d.N, 128));
    pf.end(s);
    pf.launches += 2;
    return cudaGetLastError();
}

template <typename T>
size_t Launch<T>::micro_staged_smem(int maxs) {
    const size_t need = StBytes<T>::template get<true, false>(maxs) > StBytes<T>::template get<false, true>(maxs)
                            ? StBytes<T>::template get<true, false>(maxs) : StBytes<T>::template get<false, true>(maxs);
    const size_t need2 = need > StBytes<T>::template get<false, false>(maxs) ? need : StBytes<T>::template get<false, false>(maxs);
    int dev = 0, lim = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    // the kernels' static shared memory comes on top of the dynamic part
    if (need2 + 4096 > (size_t)lim) return 0;
    constexpr int W = MICRO_ST_WPB;
    if (cudaFuncSetAttribute(k_micro_sweep_st<T, W, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)StBytes<T>::template get<true, false>(maxs)) != cudaSuccess ||
        cudaFuncSetAttribute(k_micro_sweep_st<T, W, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)StBytes<T>::template get<false, true>(maxs)) != cudaSuccess ||
        cudaFuncSetAttribute(k_micro_sweep_st<T, W, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)StBytes<T>::template get<false, false>(maxs)) != cudaSuccess)
        return 0;
    if constexpr (std::is_same<T, float>::value) {
        const int b0 = (int)StBytes<T>::template get<true, false>(maxs);
        const int b1 = (int)StBytes<T>::template get<false, true>(maxs);
        const int b2 = (int)StBytes<T>::template get<false, false>(maxs);
        constexpr auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(k_micro_sweep_st_p<W, true, false, false>, A, b0) != cudaSuccess ||
            cudaFuncSetAttribute(k_micro_sweep_st_p<W, false, true, false>, A, b1) != cudaSuccess ||
            cudaFuncSetAttribute(k_micro_sweep_st_p<W, false, false, false>, A, b2) != cudaSuccess ||
            cudaFuncSetAttribute(k_micro_sweep_st_p<W, true, false, true>, A, b0) != cudaSuccess ||
            cudaFuncSetAttribute(k_micro_sweep_st_p<W, false, true, true>, A, b1) != cudaSuccess ||
            cudaFuncSetAttribute(k_micro_sweep_st_p<W, false, false, true>, A, b2) != cudaSuccess)
            return 0;
    }
    return need2;
}

template <typename T>
cudaError_t Launch<T>::debug_micro_flux(const Dev<T>& d, cudaStream_t s, T* out) {
    dim3 grid(d.N, cdiv(d.K, 128));
    k_debug_micro_flux<T><<<grid, 128, 0, s>>>(d, out);
    return cudaGetLastError();
}

template <typename T>
int Launch<T>::coop_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_macro_coop<T>, 128, 0) != cudaSuccess) return 0;
    return n;
}

template <typename T>
cudaError_t Launch<T>::temps(const Dev<T>& d, cudaStream_t s, double* out) {
    k_temps<T><<<cdiv(d.N, 256), 256, 0, s>>>(d, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::surface(const Dev<T>& d, cudaStream_t s, const int* wall_b, int nw,
                               double p_inf, double qdyn, double Umag, double* out,
                               double* contrib, double* tot) {
    if (nw) k_surface<T><<<cdiv(nw, 128), 128, 0, s>>>(d, wall_b, nw, p_inf, qdyn, Umag, out, contrib);
    k_sum4<<<1, 256, 0, s>>>(contrib, nw, tot);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::aero(const Dev<T>& d, cudaStream_t s, const int* wall_b, int nw,
                            const double x_ref[3], double* contrib, double* tot) {
    if (nw) k_aero<T><<<cdiv(nw, 128), 128, 0, s>>>(d, wall_b, nw, x_ref[0], x_ref[1], x_ref[2], contrib);
    k_sum6<<<1, 256, 0, s>>>(contrib, nw, tot);
    return cudaGetLastError();
}

}  // namespace rk
