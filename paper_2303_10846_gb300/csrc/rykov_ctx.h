// Host-side context of librykov (shared by the translation units of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "rykov.h"
#include "rykov_launch.cuh"

namespace rk {
struct AdjState;     // adjoint workspace and solver state (adjoint.cu)
}

namespace rkh {

constexpr int MAX_BC = 64;

struct Carver {
    char* base;
    size_t off = 0;
    template <typename X>
    X* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        X* p = base ? reinterpret_cast<X*>(base + off) : nullptr;
        off += n * sizeof(X);
        return p;
    }
};

}  // namespace rkh

using rkh::Carver;
using rkh::MAX_BC;

#ifndef RK_STAGED_DEFAULT
#define RK_STAGED_DEFAULT 4
#endif

struct rk_ctx {
    int prec = RK_FP64;
    bool debug = false;
    cudaStream_t stream = nullptr;
    std::string err;
    rk_params p{};
    bool have_params = false;
    // staged inputs
    int64_t N = 0, F = 0, K = 0;
    std::vector<int64_t> fc;
    std::vector<double> fn, fa, fx, cx, cv;
    std::vector<int32_t> col;
    std::vector<double> u, w;
    int bck[MAX_BC];
    double bcv[MAX_BC * 5];
    // derived (host)
    int Kp = 0, C = 0, nnz = 0, Fi = 0, Fb = 0, nwall = 0;
    std::vector<int> slot_off, slot_face, slot_nbr, slot_left, slot_ncol, face_int, face_bnd,
        col_off, col_cell, wall_b, fc32;
    std::vector<double> slot_n;
    bool mesh_ok = false, dvs_ok = false;
    // device
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool bound = false;
    rk::Dev<double> dd{};
    rk::Dev<float> df{};
    rk::Sched sched{};
    rk::Prof prof{};
    double *stage_a = nullptr, *stage_b = nullptr;   // [N][6] staging for host inputs
    double* surf_out = nullptr;                       // [nwall][8]
    double* surf_contrib = nullptr;                   // [nwall][4]
    double* surf_tot = nullptr;                       // [4]
    double* aero_contrib = nullptr;                   // [nwall][6]
    double* aero_tot = nullptr;                       // [6]
    int* wall_b_dev = nullptr;
    void* dbg = nullptr;                              // [2][N][Kp] T (debug contexts)
    double* pin = nullptr;                            // pinned host: 16 doubles
    int64_t iter = 0;
    bool have_state = false;
    // CUDA graph of one implicit iteration (captured on a private stream, launched on
    // the caller's stream); rebuilt after anything baked into it changes
    bool use_graph = true;
    bool use_coop = false;            // cooperative launch of the macro PR-SGS (RYKOV_COOP=1)
    int use_staged = RK_STAGED_DEFAULT;   // staged micro sweeps, bit mask (RYKOV_STAGED)
    bool use_prio = true;                 // stream priorities for the graph branches (RYKOV_PRIO)
    bool use_macro32 = false;             // FP32 delta-form macro PR-SGS in mixed contexts
    bool use_pdl = false;                 // its phases with programmatic serialisation (RYKOV_PDL=1)
    bool use_packed = true;               // mixed kernels on the packed FP32 pipe (RYKOV_PACKED)
    cudaStream_t cap = nullptr, cap2 = nullptr;   // capture streams (main, side branch)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_bnd = nullptr, ev_int = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    double last_res[6] = {0, 0, 0, 0, 0, 0};
    // adjoint of the steady residual (FP64 contexts; second caller-owned workspace)
    rk::AdjState* adj = nullptr;
    int bind_gen = 0;                 // incremented by every workspace bind
    long long state_ver = 0;          // incremented by every change of the state X
};

// releases the adjoint state (adjoint.cu)
void rk_adj_release(rk_ctx* ctx);

static inline int fail(rk_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, RK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

