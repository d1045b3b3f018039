// Launch sequences of librykov, one explicit instantiation per precision
// (kern_f64.cu: double, kern_f32.cu: float).  Every function enqueues on `s` and
// returns cudaSuccess or the first launch error.
#pragma once

#include <vector>

#include "rykov_dev.cuh"

namespace rk {

// Launch accounting and optional per-class CUDA-event timing (rk_profile).
struct Prof {
    bool on = false;
    long long launches = 0;
    std::vector<cudaEvent_t> ev;      // pool, created on enable
    std::vector<int> cls;             // class of each recorded pair
    size_t used = 0;                  // events used (2 per pair)
    void begin(int c, cudaStream_t s) {
        if (!on) return;
        if (used + 2 > ev.size()) {
            size_t n = ev.size();
            ev.resize(n ? 2 * n : 1024);
            for (size_t i = n; i < ev.size(); ++i) cudaEventCreate(&ev[i]);
        }
        cudaEventRecord(ev[used], s);
        cls.push_back(c);
    }
    void end(cudaStream_t s) {
        if (!on) return;
        cudaEventRecord(ev[used + 1], s);
        used += 2;
    }
};

struct Sched {
    const int* col_cell;            // device: cells grouped by colour
    std::vector<int> col_off;       // host: colour offsets (C+1)
    int coop_grid = 0;              // blocks of the cooperative macro solve (0: per-colour launches)
    unsigned coop_extra = 0;        // test only: barrier arrivals that never come
    unsigned long long coop_limit_ns = 1000000000ull;   // bound of every barrier wait
    int maxs = 0;                   // most faces of one cell
    int staged = 0;                 // micro sweeps with staged (asynchronous) row loads:
                                    // bit 0 first sweep, bit 1 middle sweeps, bit 2 last;
                                    // bit 3: the cell's own rows by bulk copies (packed)
    int macro32 = 0;                // macro PR-SGS in FP32 delta form (mixed contexts)
    int pdl = 0;                    // its colour phases launched with programmatic
                                    // stream serialisation
    int macro_lanes = 4;            // threads per cell of the FP32 macro phases (1, 2, 4)
};

template <typename T>
struct Launch {
    static cudaError_t setup(const Dev<T>& d, cudaStream_t s);
    static cudaError_t set_state(const Dev<T>& d, cudaStream_t s, const double* prim,
                                 const double* q);
    static cudaError_t recon(const Dev<T>& d, cudaStream_t s, Prof& pf);
    static cudaError_t faces(const Dev<T>& d, cudaStream_t s, Prof& pf);   // interior + boundary
    static cudaError_t faces_interior(const Dev<T>& d, cudaStream_t s, Prof& pf);
    static cudaError_t faces_boundary(const Dev<T>& d, cudaStream_t s, Prof& pf);
    static cudaError_t fluxes(const Dev<T>& d, cudaStream_t s, Prof& pf);
    // micro flux F into res: independent of the macro solve (a parallel graph branch)
    static cudaError_t micro_flux(const Dev<T>& d, cudaStream_t s, Prof& pf);
    static cudaError_t macro(const Dev<T>& d, cudaStream_t s, const Sched& sc, int n_macro,
                             Prof& pf);
    static cudaError_t micro(const Dev<T>& d, cudaStream_t s, const Sched& sc, int n_micro,
                             Prof& pf);
    // shared memory of the staged micro sweeps for a mesh with at most maxs faces per
    // cell (0 if it exceeds the device limit); sets the kernels' attribute
    static size_t micro_staged_smem(int maxs);
    static cudaError_t debug_micro_flux(const Dev<T>& d, cudaStream_t s, T* out);
    static cudaError_t temps(const Dev<T>& d, cudaStream_t s, double* out);
    static int coop_blocks_per_sm();
    static cudaError_t surface(const Dev<T>& d, cudaStream_t s, const int* wall_b, int nw,
                               double p_inf, double qdyn, double Umag, double* out,
                               double* contrib, double* tot);
    static cudaError_t aero(const Dev<T>& d, cudaStream_t s, const int* wall_b, int nw,
                            const double x_ref[3], double* contrib, double* tot);
};

extern template struct Launch<double>;
extern template struct Launch<float>;

}  // namespace rk
