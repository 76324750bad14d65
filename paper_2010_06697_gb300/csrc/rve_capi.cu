// Host side of the C ABI declared in include/rve.h: handle lifetime, device
// workspace layout, FFT plans and tables, and the ADMM driver loop
// (Zhou & Bhattacharya, Algorithm 1: initialise, iterate Steps 1-4 on the
// device until both residuals pass, keep the state resident between solves).
//
// The iteration loop never waits on the host per iteration: chunks of
// `check_every` iterations are replayed as one CUDA graph, every kernel exits
// at once when the device-side stop flag is set, and the host reads the control
// block once per chunk.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/rve.h"
#include "rve_internal.cuh"

using admm::Ctrl;
using admm::Launch;

struct rve {
    int dim = 0, n = 0, model = 0;
    long long V = 0;
    rve_options opt{};
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev0 = nullptr, ev1 = nullptr;
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    Launch L{};
    admm::Exec E{};         // tile-table execution of this RVE alone
    const Launch* self_mem[1] = {nullptr};   // E's member list: this RVE
    unsigned char self_exact[1] = {0};
    int self_tile0[1] = {0};
    Launch* d_L = nullptr;  // device copy of L (the descriptor the tile kernels read)
    Ctrl* hctrl = nullptr;  // pinned host mirror of the control block
    bool material_set = false;
    bool fresh = true;
    int state_fp64 = 1;     // which set holds the current state
    double mu_ref = 1.0;
    int nphase = 0;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // float, double, double polish
    unsigned free_mask = 0;    // mixed control of the solve in progress (bit 3i+j: <F_ij> free)
    bool graph_free = false;   // the cached graphs contain the mixed-control kernel
    long long k = 0;        // host copy of Ctrl::k
    int last_iters = 0;
    long long launches = 0; // kernel launches issued by the running solve
    // profiling: every launch bracketed by events, per kernel class and precision
    admm::BlochWork* bloch = nullptr;  // Bloch-wave workspace (rve_bloch)
    bool prof = false;
    std::vector<cudaEvent_t> pev;
    double prof_ms[2][RVE_KCLASS_COUNT] = {};
    long long prof_n[2][RVE_KCLASS_COUNT] = {};
};

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_n(int n) {
    if (n < 4 || n > 512 || (n & 1)) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

struct Layout {
    size_t ctrl, hist, partials, phase, mat, mat32, mat32lo, desc, tiles[admm::kTileClasses];
    size_t F64[2], L64, U64[2], tw64, ksq64, N64[2], n064, Fp64, np64;
    size_t F32[2], L32, U32[2], tw32, ksq32, N32[2], n032, Fp32, np32;
    size_t total;
};

Launch geometry(int dim, int n) {
    Launch g{};
    g.dim = dim;
    g.n = n;
    g.V = dim == 3 ? (long long)n * n * n : (long long)n * n;
    admm::set_geometry(g);
    return g;
}

Layout layout(int dim, int n, int model, int precision, int max_iter) {
    Layout o{};
    const Launch g = geometry(dim, n);
    const long long V = g.V;
    const size_t nF = (size_t)dim * dim * V, nU = (size_t)dim * V;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    o.ctrl = take(sizeof(Ctrl));
    o.hist = take(sizeof(double) * admm::kHistStride * (size_t)(max_iter + 1));
    o.partials = take(sizeof(double) * admm::kPartialStride * (size_t)g.local_blocks);
    o.desc = take(sizeof(Launch));
    o.tiles[admm::kTilesLocal] = take(sizeof(int2) * (size_t)admm::tiles_local(g));
    o.tiles[admm::kTilesX] = take(sizeof(int2) * (size_t)admm::tiles_x(g));
    o.tiles[admm::kTilesAx64] = take(sizeof(int2) * (size_t)admm::tiles_ax(g, true));
    o.tiles[admm::kTilesAx32] = take(sizeof(int2) * (size_t)admm::tiles_ax(g, false));
    o.phase = take((size_t)V);
    o.mat = take(sizeof(double) * 256 * admm::kMaxParam);
    o.mat32 = take(sizeof(float) * 256 * admm::kMaxParam);
    o.mat32lo = take(sizeof(float) * 256 * admm::kMaxParam);
    const bool need64 = precision != RVE_FP32;
    const bool need32 = precision != RVE_FP64;
    const bool lce = model == admm::kLce;
    if (need64) {
        o.F64[0] = take(8 * nF);
        o.F64[1] = take(8 * nF);
        o.L64 = take(8 * nF);
        o.U64[0] = take(8 * nU);
        o.U64[1] = take(8 * nU);
        o.tw64 = take(16 * (size_t)n);
        o.ksq64 = take(8 * (size_t)n);
        if (lce) {
            o.N64[0] = take(8 * 3 * (size_t)V);
            o.N64[1] = take(8 * 3 * (size_t)V);
            o.n064 = take(8 * 3 * (size_t)V);
            o.Fp64 = take(8 * 9 * (size_t)V);
            o.np64 = take(8 * 3 * (size_t)V);
        }
    }
    if (need32) {
        o.F32[0] = take(4 * nF);
        o.F32[1] = take(4 * nF);
        o.L32 = take(4 * nF);
        o.U32[0] = take(4 * nU);
        o.U32[1] = take(4 * nU);
        o.tw32 = take(8 * (size_t)n);
        o.ksq32 = take(4 * (size_t)n);
        if (lce) {
            o.N32[0] = take(4 * 3 * (size_t)V);
            o.N32[1] = take(4 * 3 * (size_t)V);
            o.n032 = take(4 * 3 * (size_t)V);
            o.Fp32 = take(4 * 9 * (size_t)V);
            o.np32 = take(4 * 3 * (size_t)V);
        }
    }
    o.total = off;
    return o;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return RVE_E_CUDA; \
    } while (0)

int read_ctrl_on(rve* h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->hctrl, h->L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->k = h->hctrl->k;
    return RVE_OK;
}
int read_ctrl(rve* h) { return read_ctrl_on(h, h->stream); }

int write_ctrl_on(rve* h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h->L.ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    return RVE_OK;
}
int write_ctrl(rve* h) { return write_ctrl_on(h, h->stream); }

// Copy the host descriptor to the device copy the tile kernels read.
int write_desc(rve* h) {
    CK(cudaMemcpyAsync(h->d_L, &h->L, sizeof(Launch), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return RVE_OK;
}

int check_solve_args(const rve* h, const double Fbar[9], double rho, double tol) {
    if (!h || !Fbar) return RVE_E_INVALID_ARG;
    if (!h->material_set) return RVE_E_STATE;
    if (!(rho > 0) || !isfinite(rho) || isnan(tol)) return RVE_E_INVALID_ARG;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(Fbar[i])) return RVE_E_INVALID_ARG;
    const double det2 = Fbar[0] * Fbar[4] - Fbar[1] * Fbar[3];
    const double det3 = Fbar[0] * (Fbar[4] * Fbar[8] - Fbar[5] * Fbar[7]) -
                        Fbar[1] * (Fbar[3] * Fbar[8] - Fbar[5] * Fbar[6]) +
                        Fbar[2] * (Fbar[3] * Fbar[7] - Fbar[4] * Fbar[6]);
    if (!((h->dim == 2 ? det2 : det3) > 0)) return RVE_E_INVALID_ARG;
    return RVE_OK;
}

// Prepare the control block of a solve (Algorithm 1's initialisation) and, for a
// fresh state, the initial fields; everything on stream st.  Leaves the first
// precision phase ready to start (its FIRST local step not yet launched).
int begin_solve(rve* h, const double Fbar[9], double rho, double tol, cudaStream_t st) {
    const rve_options& o = h->opt;
    int rc = read_ctrl_on(h, st);
    if (rc) return rc;
    Ctrl& c = *h->hctrl;
    for (int i = 0; i < 9; ++i) c.Fbar[i] = c.Fbar_prev[i] = Fbar[i];
    c.free_mask = h->free_mask;
    c.dw_state = 0;
    c.div_given = 0;
    c.z_valid = 0;
    c.u_pair = 0;
    c.spec_have = 0;  // the spectrum kept for r_d is that of an earlier state
    c.spec_next = 0;
    c.spec_sum = 0;
    c.rho = rho;
    c.inv_rho = 1.0 / rho;
    c.mu_ref = o.mu_ref > 0 ? o.mu_ref : h->mu_ref;
    c.tol = tol;
    c.rho_kappa = o.rho_kappa;
    c.rho_tau = o.rho_tau;
    c.rho_min = o.rho_min > 0 ? o.rho_min : c.mu_ref;
    c.switch_tol = o.mixed_switch;
    c.best = INFINITY;
    c.stall = 0;
    c.k_start = c.k;
    c.k_cap = c.k + o.max_iter;
    c.done = o.max_iter > 0 ? admm::kRunning : admm::kCapped;
    c.adaptive = o.rho_policy == RVE_RHO_ADAPTIVE;
    c.rho_changed = 0;
    c.newton_cap = o.newton_max;
    for (int b = 0; b < admm::kNewtonBins; ++b) c.newton_hist[b] = 0u;
    c.hist_cap = o.max_iter + 1;
    c.local_ratio = o.local_ratio;
    c.local_fraction = o.local_fraction;
    c.newton_cap_max = o.newton_max;
    c.r_d = 0.0;  // no check yet: the first two local steps of the solve are exact
    c.rd_local = 0.0;
    c.r_l = 0.0;
    c.counter = 0;
    c.counter2 = 0;
    c.newton_max = 0;
    c.newton_fail = 0;
    const bool fp32_first = o.precision != RVE_FP64;
    c.phase_fp32 = fp32_first ? 1 : 0;
    c.newton_tol = o.newton_tol > 0 ? o.newton_tol : (fp32_first ? 1e-5 : 1e-10);
    if (write_ctrl_on(h, st)) return RVE_E_CUDA;
    CK(cudaMemcpyAsync(h->d_L, &h->L, sizeof(Launch), cudaMemcpyHostToDevice, st));
    Launch Ls = h->L;
    Ls.stream = st;
    if (h->fresh) {
        h->launches += 1;
        if (admm::launch_init(Ls, !fp32_first, o.lambda0 == RVE_LAMBDA0_ZERO) != cudaSuccess) return RVE_E_CUDA;
        h->fresh = false;
        h->state_fp64 = fp32_first ? 0 : 1;
    } else if (fp32_first && h->state_fp64) {
        h->launches += 1;
        if (admm::launch_convert(Ls, false) != cudaSuccess) return RVE_E_CUDA;
        h->state_fp64 = 0;
    }
    if (h->model == admm::kLce) {  // the time step's starting state, for the dissipation terms
        h->launches += 1;
        if (admm::launch_save_prev(Ls, h->state_fp64 != 0, st) != cudaSuccess) return RVE_E_CUDA;
    }
    return RVE_OK;
}

// The polish can start straight from the float state (admm::launch_switch_direct) for
// the elastic laws without free <F> components; the others begin it with a double local
// step, a double projection and a double fused pass from the state converted to double.
bool switch_direct_ok(const rve* h) {
    return (h->model == admm::kNeoHooke || h->model == admm::kLinear) && h->free_mask == 0;
}

// The switch of RVE_MIXED from the float phase to the double polish, on stream st.
int switch_to_double(rve* h, cudaStream_t st, bool direct) {
    Launch Ls = h->L;
    Ls.stream = st;
    h->launches += 1;
    if (!direct && admm::launch_convert(Ls, true) != cudaSuccess) return RVE_E_CUDA;
    h->state_fp64 = 1;
    h->hctrl->done = admm::kRunning;
    h->hctrl->phase_fp32 = 0;
    h->hctrl->counter = 0;
    // polish: a step of max|dF| <= 1e-7 leaves an error of about 1e-6 * 1e-7 (float
    // Hessian) + |dF|^2, i.e. ~1e-13, far below the double residual tolerance
    h->hctrl->newton_tol = h->opt.newton_tol > 0 ? h->opt.newton_tol : 1e-7;
    // the adaptive penalty acts during the float bulk; the double polish (increment form)
    // needs a constant rho, so it keeps the value reached here
    h->hctrl->adaptive = 0;
    h->hctrl->rho_changed = 0;  // a pending redo is subsumed by the polish's first local step
    h->hctrl->z_valid = 0;
    if (direct) {  // the state becomes double-words and the first x-forward pass takes r
        h->hctrl->dw_state = 1;
        h->hctrl->div_given = 1;
    }
    if (write_ctrl_on(h, st)) return RVE_E_CUDA;
    if (direct) {
        h->launches += 1;
        if (admm::launch_switch_direct(Ls, st) != cudaSuccess) return RVE_E_CUDA;
    }
    return RVE_OK;
}

int status_of(int done) {
    switch (done) {
        case admm::kConverged: return RVE_OK;
        case admm::kNumerical: return RVE_E_NUMERICAL;
        default: return RVE_E_NOT_CONVERGED;
    }
}

void fill_info(rve* h, long long k0, int fp64_iters, double ms, rve_solve_info* info) {
    const Ctrl& e = *h->hctrl;
    const int status = status_of(e.done);
    h->last_iters = (int)(e.k - k0);
    if (!info) return;
    info->iterations = h->last_iters;
    info->fp64_iterations = fp64_iters;
    info->converged = e.done == admm::kConverged;
    info->status = status;
    info->r_p = e.r_p;
    info->r_d = e.r_d;
    info->r_l = e.r_l;
    info->rho = e.rho;
    info->mu_ref = e.mu_ref;
    info->newton_max_iters = e.newton_max;
    info->newton_fail = (long long)e.newton_fail;
    info->time_ms = ms;
    info->launches = h->launches;
}

// Order the handle's stream after everything already queued on the caller's stream.
int enter(rve* h) {
    CK(cudaEventRecord(h->ev_in, h->user_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
    return RVE_OK;
}

// kernel class of FFT stage s (see rve_kernel_times)
int fft_class(int dim, int s) {
    if (dim == 3) return RVE_KCLASS_XFWD + s;
    return s == 0 ? RVE_KCLASS_XFWD : (s == 1 ? RVE_KCLASS_SOLVE : RVE_KCLASS_XINV);
}

int launches_per_iteration(const rve* h) {
    return admm::fft_stages(h->dim) + 1 + (h->opt.rho_policy == RVE_RHO_ADAPTIVE ? 1 : 0) + (h->free_mask ? 1 : 0);
}

// Mixed control: the free components of <F> for the coming projection (no-op
// without).  polish: the state is in the double-word form of the elastic laws.
cudaError_t macro_step(rve* h, bool fp64, bool polish = false) {
    if (!h->free_mask) return cudaSuccess;
    return admm::launch_macro(h->L, fp64, h->stream, polish && h->model != admm::kLce);
}

int ensure_prof_events(rve* h) {
    const size_t need = (size_t)h->opt.check_every * (admm::fft_stages(h->dim) + 3) + 2;
    while (h->pev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->pev.push_back(e);
    }
    return RVE_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// Profiled variant of one chunk: direct launches with an event after each kernel;
// only iterations that ran (before the stop flag) are accumulated.  incr: the
// double polish of RVE_MIXED (float increment projection + local with R).
int run_chunk_profiled(rve* h, bool fp64, bool incr) {
    const int S = admm::fft_stages(h->dim);
    const int per = S + 2 + 1;  // start event, S fft, local, redo
    const long long k_before = h->hctrl->k;
    const int f = fp64 ? 1 : 0;
    for (int i = 0; i < h->opt.check_every; ++i) {
        cudaEvent_t* e = &h->pev[(size_t)i * per];
        if (macro_step(h, fp64, incr) != cudaSuccess) return RVE_E_CUDA;
        CK(cudaEventRecord(e[0], h->stream));
        for (int st = 0; st < S; ++st) {
            const cudaError_t le = incr ? admm::launch_fft_incr(h->E, st) : admm::launch_fft(h->E, fp64, st);
            if (le != cudaSuccess) return RVE_E_CUDA;
            CK(cudaEventRecord(e[1 + st], h->stream));
        }
        if (admm::launch_local(h->E, fp64, false, false, incr ? 2 : 0) != cudaSuccess) return RVE_E_CUDA;
        CK(cudaEventRecord(e[1 + S], h->stream));
        if (h->opt.rho_policy == RVE_RHO_ADAPTIVE) {
            if (admm::launch_local(h->E, fp64, true, true) != cudaSuccess) return RVE_E_CUDA;
            CK(cudaEventRecord(e[2 + S], h->stream));
        }
    }
    const int rc = read_ctrl(h);
    if (rc) return rc;
    const long long ran = h->hctrl->k - k_before;
    for (long long i = 0; i < ran && i < h->opt.check_every; ++i) {
        cudaEvent_t* e = &h->pev[(size_t)i * per];
        for (int st = 0; st < S; ++st) {
            if (admm::fft_stage_empty(h->E, fp64 && !incr, st)) continue;  // folded into a fused pass
            int cls = fft_class(h->dim, st), fb = f;
            if (incr) {
                fb = 0;
                if (st == 0) cls = RVE_KCLASS_XFWD_INCR;
                if (st == S - 1) cls = RVE_KCLASS_XINV_INCR;
            }
            h->prof_ms[fb][cls] += elapsed(e[st], e[st + 1]);
            h->prof_n[fb][cls] += 1;
        }
        const int lc = incr ? RVE_KCLASS_LOCAL_R : RVE_KCLASS_LOCAL;
        h->prof_ms[f][lc] += elapsed(e[S], e[S + 1]);
        h->prof_n[f][lc] += 1;
    }
    return RVE_OK;
}

int capture_chunk(rve* h, bool fp64, bool incr, int slot) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < h->opt.check_every && e == cudaSuccess; ++i) {
        e = macro_step(h, fp64, incr);
        if (e == cudaSuccess) e = incr ? admm::launch_fft_incr(h->E) : admm::launch_fft(h->E, fp64);
        if (e == cudaSuccess) e = admm::launch_local(h->E, fp64, false, false, incr ? 2 : 0);
        if (e == cudaSuccess && h->opt.rho_policy == RVE_RHO_ADAPTIVE) e = admm::launch_local(h->E, fp64, true, true);
    }
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return RVE_E_CUDA;
    }
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[slot], g, 0);
    cudaGraphDestroy(g);
    return e3 == cudaSuccess ? RVE_OK : RVE_E_CUDA;
}

int run_phase_body(rve* h, bool fp64, bool polish, bool direct);

// Run iterations in one precision until the device sets the stop flag.  polish
// (RVE_MIXED; rho constant from the switch on): after the first step, one full double projection,
// then increment projections in float (see admm::launch_fft_incr) with the state
// of the elastic laws held as double-words; it returns to double on every exit.
int run_phase(rve* h, bool fp64, bool polish = false, bool direct = false) {
    const int rc = run_phase_body(h, fp64, polish, direct);
    if (!polish) return rc;
    if (admm::launch_polish_state(h->L, false, h->stream) != cudaSuccess) return RVE_E_CUDA;
    h->launches += 2;
    if (rc) return rc;
    return read_ctrl(h);
}

int run_phase_body(rve* h, bool fp64, bool polish, bool direct) {
    // direct: the polish's state is already in place (switch_to_double), no first steps
    if (direct) {
    } else if (h->prof) {
        if (ensure_prof_events(h)) return RVE_E_CUDA;
        const size_t last = h->pev.size() - 2;
        CK(cudaEventRecord(h->pev[last], h->stream));
        if (admm::launch_local(h->E, fp64, true, false) != cudaSuccess) return RVE_E_CUDA;
        CK(cudaEventRecord(h->pev[last + 1], h->stream));
        CK(cudaEventSynchronize(h->pev[last + 1]));
        h->prof_ms[fp64 ? 1 : 0][RVE_KCLASS_LOCAL_FIRST] += elapsed(h->pev[last], h->pev[last + 1]);
        h->prof_n[fp64 ? 1 : 0][RVE_KCLASS_LOCAL_FIRST] += 1;
    } else if (admm::launch_local(h->E, fp64, true, false) != cudaSuccess) {
        return RVE_E_CUDA;
    }
    if (!direct) h->launches += 1;
    if (polish && !direct) {
        if (macro_step(h, true) != cudaSuccess) return RVE_E_CUDA;
        if (admm::launch_fft(h->E, true) != cudaSuccess) return RVE_E_CUDA;
        if (admm::launch_local(h->E, true, false, false, 1) != cudaSuccess) return RVE_E_CUDA;
        if (admm::launch_polish_state(h->L, true, h->stream) != cudaSuccess) return RVE_E_CUDA;
        h->launches += admm::fft_stages(h->dim) + 3;
        const int rc = read_ctrl(h);
        if (rc) return rc;
        if (h->hctrl->done != admm::kRunning) return RVE_OK;
    }
    const int slot = polish ? 2 : (fp64 ? 1 : 0);
    for (;;) {
        h->launches += (long long)h->opt.check_every * launches_per_iteration(h);
        if (h->prof) {
            const int rc = run_chunk_profiled(h, fp64, polish);
            if (rc) return rc;
            if (h->hctrl->done != admm::kRunning) return RVE_OK;
            continue;
        }
        if (h->opt.use_graph) {
            if (!h->graph[slot]) {
                const int rc = capture_chunk(h, fp64, polish, slot);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(h->graph[slot], h->stream));
        } else {
            for (int i = 0; i < h->opt.check_every; ++i) {
                if (macro_step(h, fp64, polish) != cudaSuccess) return RVE_E_CUDA;
                const cudaError_t fe = polish ? admm::launch_fft_incr(h->E) : admm::launch_fft(h->E, fp64);
                if (fe != cudaSuccess) return RVE_E_CUDA;
                if (admm::launch_local(h->E, fp64, false, false, polish ? 2 : 0) != cudaSuccess) return RVE_E_CUDA;
                if (h->opt.rho_policy == RVE_RHO_ADAPTIVE &&
                    admm::launch_local(h->E, fp64, true, true) != cudaSuccess)
                    return RVE_E_CUDA;
            }
        }
        const int rc = read_ctrl(h);
        if (rc) return rc;
        if (h->hctrl->done != admm::kRunning) return RVE_OK;
    }
}

int upload_tables(rve* h) {
    const int n = h->n;
    std::vector<double> tw(2 * (size_t)n), ksq(n);
    std::vector<float> tw32(2 * (size_t)n), ksq32(n);
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < n; ++m) {
        const double a = -2.0 * pi * (double)m / (double)n;
        tw[2 * m] = cos(a);
        tw[2 * m + 1] = sin(a);
        const double s = (m == 0 || 2 * m == n) ? 0.0 : (double)n * sin(2.0 * pi * (double)m / (double)n);
        ksq[m] = s * s;
        tw32[2 * m] = (float)tw[2 * m];
        tw32[2 * m + 1] = (float)tw[2 * m + 1];
        ksq32[m] = (float)ksq[m];
    }
    if (h->L.tw64) {
        CK(cudaMemcpyAsync((void*)h->L.tw64, tw.data(), 16 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync((void*)h->L.ksq64, ksq.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    }
    if (h->L.tw32) {
        CK(cudaMemcpyAsync((void*)h->L.tw32, tw32.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync((void*)h->L.ksq32, ksq32.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return RVE_OK;
}

int check_options(const rve_options& o) {
    if (o.precision < RVE_FP64 || o.precision > RVE_FP32) return RVE_E_INVALID_ARG;
    if (o.rho_policy != RVE_RHO_FIXED && o.rho_policy != RVE_RHO_ADAPTIVE) return RVE_E_INVALID_ARG;
    if (o.lambda0 != RVE_LAMBDA0_STRESS && o.lambda0 != RVE_LAMBDA0_ZERO) return RVE_E_INVALID_ARG;
    if (o.max_iter < 0 || o.max_iter > 10000000) return RVE_E_INVALID_ARG;
    if (o.newton_max < 1 || o.newton_max > 1000) return RVE_E_INVALID_ARG;
    if (!(o.newton_tol >= 0) || !(o.rho_kappa > 1) || !(o.rho_tau > 1) || !(o.rho_min >= 0)) return RVE_E_INVALID_ARG;
    if (!(o.mu_ref >= 0) || !(o.mixed_switch >= 0)) return RVE_E_INVALID_ARG;
    if (o.check_every < 1 || o.check_every > 4096) return RVE_E_INVALID_ARG;
    if (!(o.local_ratio >= 0) || !(o.local_ratio <= 1e6)) return RVE_E_INVALID_ARG;
    if (!(o.local_fraction >= 0) || !(o.local_fraction <= 1)) return RVE_E_INVALID_ARG;
    return RVE_OK;
}

int create_common(rve_t* out, int dim, int n, int model, const rve_options* opt, void* stream, void* ws,
                  size_t bytes) {
    if (!out) return RVE_E_INVALID_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !valid_n(n)) return RVE_E_INVALID_ARG;
    if (model != RVE_NEOHOOKE && model != RVE_LINEAR && model != RVE_LCE) return RVE_E_INVALID_ARG;
    if (model == RVE_LCE && dim != 3) return RVE_E_INVALID_ARG;
    rve_options o;
    rve_default_options(&o);
    if (opt) o = *opt;
    if (check_options(o)) return RVE_E_INVALID_ARG;
    const Layout lay = layout(dim, n, model, o.precision, o.max_iter);
    if (ws && (bytes < lay.total || ((uintptr_t)ws % kAlign) != 0)) return RVE_E_OOM;

    rve* h = new (std::nothrow) rve();
    if (!h) return RVE_E_OOM;
    h->dim = dim;
    h->n = n;
    h->model = model;
    h->V = dim == 3 ? (long long)n * n * n : (long long)n * n;
    h->opt = o;
    h->user_stream = (cudaStream_t)stream;
    auto fail = [&](int code) {
        rve_destroy(h);
        return code;
    };
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RVE_E_CUDA);
    if (cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(RVE_E_CUDA);
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) return fail(RVE_E_CUDA);
    if (cudaMallocHost((void**)&h->hctrl, sizeof(Ctrl)) != cudaSuccess) return fail(RVE_E_CUDA);
    memset(h->hctrl, 0, sizeof(Ctrl));
    if (ws) {
        h->ws = (unsigned char*)ws;
        h->ws_bytes = bytes;
    } else {
        if (cudaMalloc((void**)&h->ws, lay.total) != cudaSuccess) return fail(RVE_E_OOM);
        h->own_ws = true;
        h->ws_bytes = lay.total;
    }
    if (enter(h)) return fail(RVE_E_CUDA);
    if (cudaMemsetAsync(h->ws, 0, lay.total, h->stream) != cudaSuccess) return fail(RVE_E_CUDA);

    Launch& L = h->L;
    unsigned char* b = h->ws;
    L.stream = h->stream;
    L.dim = dim;
    L.n = n;
    L.model = model;
    L.V = h->V;
    admm::set_geometry(L);
    L.ctrl = (Ctrl*)(b + lay.ctrl);
    L.hist = (double*)(b + lay.hist);
    L.partials = (double*)(b + lay.partials);
    L.phase = (const uint8_t*)(b + lay.phase);
    L.mat = (const double*)(b + lay.mat);
    L.mat32 = (const float*)(b + lay.mat32);
    L.mat32lo = (const float*)(b + lay.mat32lo);
    L.nparam = 2;
    const bool lce = model == admm::kLce;
    if (o.precision != RVE_FP32) {
        L.F64[0] = (double*)(b + lay.F64[0]);
        L.F64[1] = (double*)(b + lay.F64[1]);
        L.L64 = (double*)(b + lay.L64);
        L.U64[0] = (double*)(b + lay.U64[0]);
        L.U64[1] = (double*)(b + lay.U64[1]);
        L.tw64 = (const double2*)(b + lay.tw64);
        L.ksq64 = (const double*)(b + lay.ksq64);
        if (lce) {
            L.N64[0] = (double*)(b + lay.N64[0]);
            L.N64[1] = (double*)(b + lay.N64[1]);
            L.n0_64 = (const double*)(b + lay.n064);
            L.Fp64 = (double*)(b + lay.Fp64);
            L.np64 = (double*)(b + lay.np64);
        }
    }
    if (o.precision != RVE_FP64) {
        L.F32[0] = (float*)(b + lay.F32[0]);
        L.F32[1] = (float*)(b + lay.F32[1]);
        L.L32 = (float*)(b + lay.L32);
        L.U32[0] = (float*)(b + lay.U32[0]);
        L.U32[1] = (float*)(b + lay.U32[1]);
        L.tw32 = (const float2*)(b + lay.tw32);
        L.ksq32 = (const float*)(b + lay.ksq32);
        if (lce) {
            L.N32[0] = (float*)(b + lay.N32[0]);
            L.N32[1] = (float*)(b + lay.N32[1]);
            L.n0_32 = (const float*)(b + lay.n032);
            L.Fp32 = (float*)(b + lay.Fp32);
            L.np32 = (float*)(b + lay.np32);
        }
    }
    if (o.precision == RVE_MIXED) {
        L.R32 = L.F32[0];
        L.S32 = L.U32[0];
        L.D32 = L.U32[1];
        L.LH32 = L.L32;
        L.LL32 = L.F32[1];
        // the float phase's solved spectrum (3 V/2 complex = 12 V bytes) and the z pass's
        // tile sums for r_d live in the double u~ buffer 0 (24 V bytes), idle until the polish
        if (dim == 3 && (n == 128 || n == 256 || n == 512) && L.model == admm::kNeoHooke && o.local_ratio == 0.0 &&
            o.local_fraction == 0.0) {
            unsigned char* u0 = reinterpret_cast<unsigned char*>(L.U64[0]);
            L.Sprev = reinterpret_cast<float*>(u0);
            L.nz = admm::tiles_ax(L, false);
            L.zpart = reinterpret_cast<double*>(u0 + align_up(sizeof(float) * 3 * (size_t)L.V));
        }
    }
    if (L.plan.np_half < 0 || L.plan.np_full < 0) return fail(RVE_E_INVALID_ARG);
    if (admm::prepare_fft_kernels(n) != cudaSuccess) return fail(RVE_E_CUDA);
    // single-RVE execution: descriptor and tile tables (RVE index 0) in the workspace
    h->d_L = (Launch*)(b + lay.desc);
    {
        std::vector<int2> t;
        admm::Exec& E = h->E;
        E.stream = h->stream;
        E.rep = &h->L;
        E.rds = h->d_L;
        const int counts[admm::kTileClasses] = {admm::tiles_local(L), admm::tiles_x(L), admm::tiles_ax(L, true),
                                                admm::tiles_ax(L, false)};
        for (int c = 0; c < admm::kTileClasses; ++c) {
            t.resize(counts[c]);
            for (int i = 0; i < counts[c]; ++i) t[i] = make_int2(0, i);
            int2* dst = (int2*)(b + lay.tiles[c]);
            if (cudaMemcpyAsync(dst, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess)
                return fail(RVE_E_CUDA);
            E.tiles[c] = dst;
            E.ntiles[c] = counts[c];
        }
        for (int f = 0; f < 2; ++f) {
            E.smem_x[f] = admm::smem_x_bytes(L, f == 1);
            E.smem_a[f] = admm::smem_a_bytes(L, f == 1);
        }
        E.uniform_n = n;
        E.uniform_geom = 1;
        E.exact_local = (o.local_ratio == 0.0 && o.local_fraction == 0.0) ? 1 : 0;
        h->self_mem[0] = &h->L;
        h->self_exact[0] = (unsigned char)E.exact_local;
        E.nmem = 1;
        E.mem = h->self_mem;
        E.mem_exact = h->self_exact;
        E.mem_tile0 = h->self_tile0;
    }
    h->state_fp64 = o.precision == RVE_FP64 ? 1 : 0;
    h->hctrl->hist_cap = o.max_iter + 1;
    if (write_ctrl(h)) return fail(RVE_E_CUDA);
    if (upload_tables(h)) return fail(RVE_E_CUDA);
    *out = h;
    return RVE_OK;
}

// The iteration loop of one solve (Algorithm 1 for one load step) with the mixed
// control mask already in h->free_mask.
int solve_body(rve* h, const double Fbar[9], double rho, double tol, rve_solve_info* info) {
    int rc;
    const rve_options& o = h->opt;
    if (enter(h)) return RVE_E_CUDA;
    h->launches = 0;
    CK(cudaEventRecord(h->ev0, h->stream));
    rc = begin_solve(h, Fbar, rho, tol, h->stream);
    if (rc) return rc;
    const bool fp32_first = o.precision != RVE_FP64;
    const long long k0 = h->hctrl->k;
    int fp64_iters = 0;
    if (h->hctrl->done == admm::kRunning) {
        rc = run_phase(h, !fp32_first);
        if (rc) return rc;
        if (o.precision == RVE_MIXED && h->hctrl->done == admm::kSwitch) {
            const long long ksw = h->hctrl->k;
            const bool direct = switch_direct_ok(h);
            if (switch_to_double(h, h->stream, direct)) return RVE_E_CUDA;
            rc = run_phase(h, true, true, direct);
            if (rc) return rc;
            fp64_iters = (int)(h->hctrl->k - ksw);
        } else if (o.precision == RVE_FP64) {
            fp64_iters = (int)(h->hctrl->k - k0);
        }
    }
    CK(cudaEventRecord(h->ev1, h->stream));
    CK(cudaEventSynchronize(h->ev1));
    if (read_ctrl(h)) return RVE_E_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    fill_info(h, k0, fp64_iters, ms, info);
    return status_of(h->hctrl->done);
}

}  // namespace

extern "C" {

void rve_default_options(rve_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = RVE_FP64;
    o->rho_policy = RVE_RHO_FIXED;
    o->lambda0 = RVE_LAMBDA0_STRESS;
    o->max_iter = 1000;
    o->newton_max = 30;
    o->newton_tol = 0.0;
    o->rho_kappa = 1.3;
    o->rho_tau = 10.0;
    o->rho_min = 0.0;
    o->mu_ref = 0.0;
    o->mixed_switch = 3e-7;
    o->check_every = 16;
    o->use_graph = 1;
    o->local_ratio = 0.0;
    o->local_fraction = 0.0;
}

size_t rve_workspace_bytes(int dim, int n, int model, const rve_options* opt) {
    if ((dim != 2 && dim != 3) || !valid_n(n)) return 0;
    rve_options o;
    rve_default_options(&o);
    if (opt) o = *opt;
    if (check_options(o)) return 0;
    return layout(dim, n, model, o.precision, o.max_iter).total;
}

int rve_create(rve_t* out, int dim, int n, int model, const rve_options* opt, void* cuda_stream) {
    return create_common(out, dim, n, model, opt, cuda_stream, nullptr, 0);
}

int rve_create_in(rve_t* out, int dim, int n, int model, const rve_options* opt, void* cuda_stream,
                  void* device_workspace, size_t bytes) {
    if (!device_workspace || reinterpret_cast<uintptr_t>(device_workspace) % kAlign != 0) return RVE_E_INVALID_ARG;
    return create_common(out, dim, n, model, opt, cuda_stream, device_workspace, bytes);
}

void rve_destroy(rve_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < 3; ++i)
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    if (h->bloch) admm::bloch_free(h->bloch);
    if (h->hctrl) cudaFreeHost(h->hctrl);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// out[i] = (float)in[i] (round to nearest, as the host conversion): the float copy of the
// reference directors of a handle that holds both precisions, made from the double copy
// already on the device instead of a host conversion and a second upload.
__global__ void k_narrow(const double* __restrict__ in, float* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// Voxel count of each phase id; false if some voxel's id is >= nphase.  For up to 8
// phases it compares 8 voxels at a time (SWAR: a byte of x = w ^ (p in every byte) is zero
// exactly where the voxel has phase p; the per-byte nonzero test (x | ((x & 0x7f..) +
// 0x7f..)) & 0x80.. carries nothing across bytes, and a multiply sums the matches); every
// voxel is valid exactly when the counts add up to V.  More phases: four counter banks.
// (One counter update per voxel serialises on its own store: milliseconds per call at 128^3.)
static bool phase_histogram(const uint8_t* phase, long long V, int nphase, long long* count) {
    if (nphase <= 8) {
        const uint64_t lo7 = 0x7f7f7f7f7f7f7f7full, hi = 0x8080808080808080ull, ones = 0x0101010101010101ull;
        long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        long long v = 0;
        for (; v + 8 <= V; v += 8) {
            uint64_t w;
            memcpy(&w, phase + v, 8);
            for (int p = 0; p < nphase; ++p) {
                const uint64_t x = w ^ (ones * (uint64_t)p);
                c[p] += (long long)((((~(x | ((x & lo7) + lo7)) & hi) >> 7) * ones) >> 56);
            }
        }
        for (; v < V; ++v)
            if (phase[v] < nphase) c[phase[v]]++;
        long long tot = 0;
        for (int p = 0; p < nphase; ++p) {
            count[p] = c[p];
            tot += c[p];
        }
        return tot == V;
    }
    std::vector<long long> bank(4 * 256, 0);
    unsigned bad = 0;
    long long v = 0;
    for (; v + 4 <= V; v += 4) {
        const uint8_t a = phase[v], b = phase[v + 1], c = phase[v + 2], d = phase[v + 3];
        bad |= (unsigned)(a >= nphase) | (unsigned)(b >= nphase) | (unsigned)(c >= nphase) | (unsigned)(d >= nphase);
        bank[a]++;
        bank[256 + b]++;
        bank[512 + c]++;
        bank[768 + d]++;
    }
    for (; v < V; ++v) {
        bad |= (unsigned)(phase[v] >= nphase);
        bank[phase[v]]++;
    }
    for (int k = 0; k < 4; ++k)
        for (int p = 0; p < 256; ++p) count[p] += bank[k * 256 + p];
    return bad == 0;
}

int rve_set_material(rve_t h, const uint8_t* phase, int nphase, const double* params, int nparam,
                     const double* n0) {
    if (!h || !phase || !params || nphase < 1 || nphase > 256 || nparam < 2 || nparam > admm::kMaxParam)
        return RVE_E_INVALID_ARG;
    const bool lce = h->model == RVE_LCE;
    if (lce && (nparam < 5 || !n0)) return RVE_E_INVALID_ARG;
    std::vector<long long> count(256, 0);
    if (!phase_histogram(phase, h->V, nphase, count.data())) return RVE_E_INVALID_ARG;
    std::vector<double> tab(256 * (size_t)admm::kMaxParam, 0.0);
    double musum = 0.0;
    const double inc0 = lce && nparam > 7 ? params[7] : 0.0;  // every phase the same network
    for (int p = 0; p < nphase; ++p) {
        const double mu = params[p * nparam + 0], lam = params[p * nparam + 1];
        if (!(mu > 0) || !(lam >= 0) || !isfinite(mu) || !isfinite(lam)) return RVE_E_INVALID_ARG;
        double* row = &tab[p * admm::kMaxParam];
        for (int q = 0; q < (lce ? 5 : nparam); ++q) row[q] = params[p * nparam + q];
        if (lce && nparam > 5) {  // nu_F/dt and nu_n/dt of the dissipation (default 0)
            row[8] = params[p * nparam + 5];
            row[9] = nparam > 6 ? params[p * nparam + 6] : 0.0;
            if (!(row[8] >= 0) || !(row[9] >= 0) || !isfinite(row[8]) || !isfinite(row[9])) return RVE_E_INVALID_ARG;
        }
        if (lce && nparam > 7) {  // incompressible network: det F = 1 by the local step's multiplier
            const double inc = params[p * nparam + 7];
            if ((inc != 0.0 && inc != 1.0) || inc != inc0) return RVE_E_INVALID_ARG;
        }
        if (lce) {
            // {mu, lam, r, alpha, kappa_F}; derived a = mu r^{1/3}, c1, c2 of the m = F^T n form
            const double r = row[2], alpha = row[3], kap = row[4];
            if (!(r > 0) || !(alpha >= 0) || !(kap >= 0) || !isfinite(r) || !isfinite(alpha) || !isfinite(kap))
                return RVE_E_INVALID_ARG;
            const double r13 = cbrt(r);
            row[5] = mu * r13;
            row[6] = mu * (alpha - r13 * (1.0 - 1.0 / r));
            row[7] = mu * alpha;
        }
        musum += mu * (double)count[p];
    }
    std::vector<float> n0f;
    if (lce) {
        const long long V = h->V;
        for (long long v = 0; v < V; ++v) {
            const double a = n0[v], b = n0[V + v], c = n0[2 * V + v];
            const double nn = a * a + b * b + c * c;
            if (!isfinite(nn) || fabs(nn - 1.0) > 1e-6) return RVE_E_INVALID_ARG;
        }
        if (h->L.n0_32 && !h->L.n0_64) {  // float-only handle: narrowed here, else on the device
            n0f.resize(3 * (size_t)V);
            for (size_t i = 0; i < n0f.size(); ++i) n0f[i] = (float)n0[i];
        }
    }
    if (enter(h)) return RVE_E_CUDA;
    CK(cudaMemcpyAsync((void*)h->L.phase, phase, (size_t)h->V, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync((void*)h->L.mat, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    std::vector<float> tab32(tab.size()), tab32lo(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) {
        tab32[i] = (float)tab[i];
        tab32lo[i] = (float)(tab[i] - (double)tab32[i]);
    }
    CK(cudaMemcpyAsync((void*)h->L.mat32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync((void*)h->L.mat32lo, tab32lo.data(), tab32lo.size() * sizeof(float), cudaMemcpyHostToDevice,
                       h->stream));
    if (lce && h->L.n0_64)
        CK(cudaMemcpyAsync((void*)h->L.n0_64, n0, 3 * (size_t)h->V * 8, cudaMemcpyHostToDevice, h->stream));
    if (lce && h->L.n0_32 && h->L.n0_64) {
        const long long n3 = 3 * h->V;
        const int blocks = (int)std::min<long long>((n3 + 255) / 256, 152LL * 8);
        k_narrow<<<blocks, 256, 0, h->stream>>>(h->L.n0_64, (float*)h->L.n0_32, n3);
        CK(cudaGetLastError());
    } else if (lce && h->L.n0_32) {
        CK(cudaMemcpyAsync((void*)h->L.n0_32, n0f.data(), n0f.size() * 4, cudaMemcpyHostToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->L.nparam = admm::kMaxParam;
    if (lce) {  // the kernels of the incompressible network are their own instances
        const int m = inc0 != 0.0 ? admm::kLceInc : admm::kLce;
        if (m != h->L.model)
            for (int i = 0; i < 3; ++i)
                if (h->graph[i]) {
                    cudaGraphExecDestroy(h->graph[i]);
                    h->graph[i] = nullptr;
                }
        h->L.model = m;
    }
    h->nphase = nphase;
    h->mu_ref = musum / (double)h->V;
    h->material_set = true;
    h->fresh = true;
    return RVE_OK;
}

int rve_reset(rve_t h) {
    if (!h) return RVE_E_INVALID_ARG;
    h->fresh = true;
    return RVE_OK;
}

int rve_solve(rve_t h, const double Fbar[9], double rho, double tol, rve_solve_info* info) {
    return rve_solve_mixed(h, Fbar, 0u, rho, tol, info);
}

int rve_solve_mixed(rve_t h, const double Fbar[9], unsigned free_mask, double rho, double tol,
                    rve_solve_info* info) {
    int rc = check_solve_args(h, Fbar, rho, tol);
    if (rc) return rc;
    unsigned allowed = 0;
    for (int i = 0; i < h->dim; ++i)
        for (int j = 0; j < h->dim; ++j) allowed |= 1u << (3 * i + j);
    if (free_mask & ~allowed) return RVE_E_INVALID_ARG;
    if ((free_mask != 0) != h->graph_free) {  // the cached iteration graphs change shape
        for (int i = 0; i < 3; ++i)
            if (h->graph[i]) {
                cudaGraphExecDestroy(h->graph[i]);
                h->graph[i] = nullptr;
            }
        h->graph_free = free_mask != 0;
    }
    h->free_mask = free_mask;
    rc = solve_body(h, Fbar, rho, tol, info);
    h->free_mask = 0;
    return rc;
}

int rve_solve_path(rve_t h, const double* Fbars, int steps, unsigned free_mask, double rho, double tol,
                   double* S_out, double* Fbar_out, rve_solve_info* infos) {
    if (!h || !Fbars || steps < 1) return RVE_E_INVALID_ARG;
    double prev[9];
    int status = RVE_OK;
    for (int s = 0; s < steps; ++s) {
        double Fb[9];
        for (int i = 0; i < 9; ++i)  // free components start from the previous step's result
            Fb[i] = (s > 0 && ((free_mask >> i) & 1u)) ? prev[i] : Fbars[9 * s + i];
        rve_solve_info info{};
        const int rc = rve_solve_mixed(h, Fb, free_mask, rho, tol, &info);
        if (rc != RVE_OK && rc != RVE_E_NOT_CONVERGED) return rc;
        if (rc != RVE_OK) status = rc;
        if (infos) infos[s] = info;
        double S[9];
        int e = rve_stress(h, S);
        if (e) return e;
        if ((e = rve_macro_gradient(h, prev))) return e;
        for (int i = 0; i < 9; ++i) {
            if (S_out) S_out[9 * s + i] = S[i];
            if (Fbar_out) Fbar_out[9 * s + i] = prev[i];
        }
    }
    return status;
}

int rve_bloch(rve_t h, const int k[3], const double* p0, double rho, double tol, int max_iter, double* p_out,
              double* hist, rve_bloch_info* info) {
    if (!h || !k || !p0 || !(rho > 0) || !isfinite(rho) || max_iter < 1 || !(tol == tol)) return RVE_E_INVALID_ARG;
    if (h->model != RVE_NEOHOOKE && h->model != RVE_LINEAR) return RVE_E_INVALID_ARG;
    bool wide = false;
    for (int j = 0; j < h->dim; ++j) {
        if (k[j] == 0) return RVE_E_INVALID_ARG;
        wide = wide || k[j] > 1 || k[j] < -1;
    }
    if (!wide) return RVE_E_INVALID_ARG;
    if (!h->material_set || h->fresh) return RVE_E_STATE;
    if (enter(h)) return RVE_E_CUDA;
    if (read_ctrl(h)) return RVE_E_CUDA;  // the resident state's parity
    admm::BlochArgs a{};
    a.dim = h->dim;
    a.n = h->n;
    a.V = h->V;
    a.model = h->model;
    const int par = (int)(h->k & 1);
    a.F_fp64 = h->state_fp64 != 0;
    a.F = a.F_fp64 ? (const void*)h->L.F64[par] : (const void*)h->L.F32[par];
    a.phase = h->L.phase;
    a.mat = h->L.mat;
    a.nparam = h->L.nparam;
    for (int j = 0; j < 3; ++j) a.k[j] = j < h->dim ? k[j] : 1;
    a.rho = rho;
    a.tol = tol;
    a.mu_ref = h->opt.mu_ref > 0 ? h->opt.mu_ref : h->mu_ref;
    a.adaptive = h->opt.rho_policy == RVE_RHO_ADAPTIVE;
    a.float_bulk = h->opt.precision != RVE_FP64;
    a.promote = h->opt.precision == RVE_MIXED;
    a.rho_kappa = h->opt.rho_kappa;
    a.rho_tau = h->opt.rho_tau;
    a.rho_min = h->opt.rho_min;
    a.max_iter = max_iter;
    a.check_every = h->opt.check_every;
    a.p0 = p0;
    a.p_out = p_out;
    a.hist_out = hist;
    a.stream = h->stream;
    admm::BlochResult r{};
    const int rc = admm::bloch_run(&h->bloch, a, &r);
    if (info) {
        info->iterations = r.iterations;
        info->converged = r.converged;
        info->beta = r.beta;
        info->rayleigh = r.rayleigh;
        info->r_p = r.r_p;
        info->r_d = r.r_d;
        info->time_ms = r.time_ms;
        info->launches = r.launches;
        info->fail = r.fail;
        info->rho = r.rho;
        info->float_iterations = r.float_iterations;
    }
    return rc;
}

int rve_macro_gradient(rve_t h, double F[9]) {
    if (!h || !F) return RVE_E_INVALID_ARG;
    if (enter(h)) return RVE_E_CUDA;
    if (read_ctrl(h)) return RVE_E_CUDA;
    for (int i = 0; i < 9; ++i) F[i] = h->hctrl->Fbar[i];
    return RVE_OK;
}

int rve_stress(rve_t h, double S[9]) {
    if (!h || !S) return RVE_E_INVALID_ARG;
    if (!h->material_set) return RVE_E_STATE;
    if (enter(h)) return RVE_E_CUDA;
    if (admm::launch_stress(h->L, h->state_fp64 != 0) != cudaSuccess) return RVE_E_CUDA;
    if (read_ctrl(h)) return RVE_E_CUDA;
    for (int i = 0; i < 9; ++i) S[i] = h->hctrl->stress[i];
    return RVE_OK;
}

int rve_mean_lambda(rve_t h, double Lm[9]) {
    if (!h || !Lm) return RVE_E_INVALID_ARG;
    if (!h->material_set) return RVE_E_STATE;
    if (enter(h)) return RVE_E_CUDA;
    if (admm::launch_stress(h->L, h->state_fp64 != 0) != cudaSuccess) return RVE_E_CUDA;
    if (read_ctrl(h)) return RVE_E_CUDA;
    for (int i = 0; i < 9; ++i) Lm[i] = h->hctrl->lam_mean[i];
    return RVE_OK;
}

static int field_ptr(rve_t h, int which, void** ptr, size_t* count) {
    const long long V = h->V;
    const int par = (int)(h->k & 1);
    const bool f64 = h->state_fp64 != 0;
    switch (which) {
        case RVE_FIELD_F:
            *ptr = f64 ? (void*)h->L.F64[par] : (void*)h->L.F32[par];
            *count = (size_t)h->dim * h->dim * V;
            return RVE_OK;
        case RVE_FIELD_LAMBDA:
            *ptr = f64 ? (void*)h->L.L64 : (void*)h->L.L32;
            *count = (size_t)h->dim * h->dim * V;
            return RVE_OK;
        case RVE_FIELD_U:
            *ptr = f64 ? (void*)h->L.U64[par] : (void*)h->L.U32[par];
            *count = (size_t)h->dim * V;
            return RVE_OK;
        case RVE_FIELD_N:
            if (h->model != RVE_LCE) return RVE_E_INVALID_ARG;
            *ptr = f64 ? (void*)h->L.N64[par] : (void*)h->L.N32[par];
            *count = 3 * (size_t)V;
            return RVE_OK;
        default: return RVE_E_INVALID_ARG;
    }
}

int rve_get_field(rve_t h, int which, double* out) {
    if (!h || !out) return RVE_E_INVALID_ARG;
    void* p;
    size_t cnt;
    int rc = field_ptr(h, which, &p, &cnt);
    if (rc) return rc;
    if (enter(h)) return RVE_E_CUDA;
    if (h->state_fp64) {
        CK(cudaMemcpyAsync(out, p, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> tmp(cnt);
        CK(cudaMemcpyAsync(tmp.data(), p, cnt * 4, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (size_t i = 0; i < cnt; ++i) out[i] = tmp[i];
    }
    return RVE_OK;
}

int rve_set_field(rve_t h, int which, const double* in) {
    if (!h || !in) return RVE_E_INVALID_ARG;
    void* p;
    size_t cnt;
    int rc = field_ptr(h, which, &p, &cnt);
    if (rc) return rc;
    for (size_t i = 0; i < cnt; ++i)
        if (!isfinite(in[i])) return RVE_E_INVALID_ARG;
    if (enter(h)) return RVE_E_CUDA;
    if (h->state_fp64) {
        CK(cudaMemcpyAsync(p, in, cnt * 8, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> tmp(cnt);
        for (size_t i = 0; i < cnt; ++i) tmp[i] = (float)in[i];
        CK(cudaMemcpyAsync(p, tmp.data(), cnt * 4, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    h->fresh = false;
    return RVE_OK;
}

int rve_history(rve_t h, double* rp, double* rd, double* rho, int cap) {
    if (!h || cap < 0) return RVE_E_INVALID_ARG;
    int cnt = h->last_iters < cap ? h->last_iters : cap;
    if (cnt > h->opt.max_iter + 1) cnt = h->opt.max_iter + 1;
    if (cnt <= 0) return 0;
    constexpr int S = admm::kHistStride;
    std::vector<double> tmp(S * (size_t)cnt);
    if (enter(h)) return RVE_E_CUDA;
    CK(cudaMemcpyAsync(tmp.data(), h->L.hist, tmp.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < cnt; ++i) {
        if (rp) rp[i] = tmp[S * i];
        if (rd) rd[i] = tmp[S * i + 1];
        if (rho) rho[i] = tmp[S * i + 2];
    }
    return cnt;
}

int rve_history_local(rve_t h, double* r_l, int cap) {
    if (!h || !r_l || cap < 0) return RVE_E_INVALID_ARG;
    int cnt = h->last_iters < cap ? h->last_iters : cap;
    if (cnt > h->opt.max_iter + 1) cnt = h->opt.max_iter + 1;
    if (cnt <= 0) return 0;
    constexpr int S = admm::kHistStride;
    std::vector<double> tmp(S * (size_t)cnt);
    if (enter(h)) return RVE_E_CUDA;
    CK(cudaMemcpyAsync(tmp.data(), h->L.hist, tmp.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < cnt; ++i) r_l[i] = tmp[S * i + 3];
    return cnt;
}

int rve_set_profiling(rve_t h, int on) {
    if (!h) return RVE_E_INVALID_ARG;
    h->prof = on != 0;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < RVE_KCLASS_COUNT; ++c) {
            h->prof_ms[f][c] = 0.0;
            h->prof_n[f][c] = 0;
        }
    return RVE_OK;
}

int rve_kernel_times(rve_t h, int fp64, double* ms, long long* launches, int cap) {
    if (!h || !ms || !launches || cap < RVE_KCLASS_COUNT) return RVE_E_INVALID_ARG;
    const int f = fp64 ? 1 : 0;
    for (int c = 0; c < RVE_KCLASS_COUNT; ++c) {
        ms[c] = h->prof_ms[f][c];
        launches[c] = h->prof_n[f][c];
    }
    return RVE_KCLASS_COUNT;
}

const char* rve_strerror(int code) {
    switch (code) {
        case RVE_OK: return "ok";
        case RVE_E_INVALID_ARG: return "invalid argument";
        case RVE_E_OOM: return "out of device memory or workspace too small";
        case RVE_E_NOT_CONVERGED: return "not converged within max_iter";
        case RVE_E_NUMERICAL: return "numerical failure (non-finite residual)";
        case RVE_E_CUDA: return "CUDA runtime error";
        case RVE_E_BUSY: return "busy: no free slot";
        case RVE_E_STATE: return "call out of order (material not set)";
        case RVE_E_NOT_FOUND: return "unknown ticket";
        default: return "unknown status";
    }
}

}  // extern "C"

// ================================================================== batches and serving
//
// Engine: RVE solves in flight on one stream.  Members sit in descriptor slots;
// members with the same (dimension, model, precision stage) form a run whose
// per-iteration passes are single persistent launches over the run's tile
// table, replayed as CUDA graphs of check_every iterations.  add() starts a
// member (its first local step on its own tiles); tick() runs one chunk of every
// run, reads every running member's stop flag, moves members of RVE_MIXED to the
// double polish and reports finished members.  Membership changes rebuild the
// affected tile tables (and graphs).  Used by rve_batch_solve (add all, tick
// until empty) and by the server (admit whenever memory frees up).

namespace {

__global__ void k_gather_status(const Launch* __restrict__ rds, const int* __restrict__ slots, int count,
                                long long* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const Ctrl* c = rds[slots[i]].ctrl;
        out[2 * i] = c->done;
        out[2 * i + 1] = c->k;
    }
}

enum Stage : int { kStageF32 = 0, kStageF64 = 1, kStagePolish = 2 };

struct BatchRun {  // members of one (dim, model, stage) still iterating
    std::vector<int> active;  // slots
    admm::Exec E{};
    int stage = 0;                      // precision stage of the run (enum Stage)
    std::vector<const Launch*> mem;     // E's member list in local-tile order: the members
    std::vector<unsigned char> mem_exact;  // without a lean local kernel first (lean_local)
    std::vector<int> mem_tile0;
    int2* d_tiles[admm::kTileClasses] = {};
    int cap[admm::kTileClasses] = {};
    cudaGraphExec_t graph = nullptr;
    bool dirty = true;
};

struct Member {
    rve* h = nullptr;
    int stage = 0;
    long long k0 = 0, ksw = -1;
    bool running = false;
};

// Members share a run (one launch per pass) by dimension, model, precision stage and
// size class: 3D cells of N = 128, 256 or 512 form runs of their own, so that their
// launches use the fixed-length FFT kernels of that N (a run of mixed sizes takes the
// general kernels); every other size goes to one shared run.
using RunKey = std::tuple<int, int, int, int>;
int size_class(const rve* h) {
    return (h->dim == 3 && (h->n == 128 || h->n == 256 || h->n == 512)) ? h->n : 0;
}

struct Engine {
    cudaStream_t stream = nullptr;
    Launch* d_rds = nullptr;
    int cap = 0;
    int* d_slots = nullptr;
    long long* d_status = nullptr;
    long long* h_status = nullptr;
    int* h_slots = nullptr;
    std::vector<Member> mem;  // by slot
    std::vector<int> free_slots;
    std::map<RunKey, BatchRun> runs;
};

void engine_free(Engine& E) {
    if (E.stream) cudaStreamSynchronize(E.stream);
    for (auto& kv : E.runs) {
        if (kv.second.graph) cudaGraphExecDestroy(kv.second.graph);
        for (int c = 0; c < admm::kTileClasses; ++c)
            if (kv.second.d_tiles[c]) cudaFree(kv.second.d_tiles[c]);
    }
    E.runs.clear();
    if (E.d_rds) cudaFree(E.d_rds);
    if (E.d_slots) cudaFree(E.d_slots);
    if (E.d_status) cudaFree(E.d_status);
    if (E.h_status) cudaFreeHost(E.h_status);
    if (E.h_slots) cudaFreeHost(E.h_slots);
    E.d_rds = nullptr;
    E.d_slots = nullptr;
    E.d_status = nullptr;
    E.h_status = nullptr;
    E.h_slots = nullptr;
    E.cap = 0;
}

int engine_reserve(Engine& E, int need) {
    if (need <= E.cap) return RVE_OK;
    int cap = std::max(need, std::max(16, 2 * E.cap));
    Launch* rds = nullptr;
    int* dsl = nullptr;
    long long *dst = nullptr, *hst = nullptr;
    int* hsl = nullptr;
    if (cudaMalloc((void**)&rds, sizeof(Launch) * cap) != cudaSuccess) return RVE_E_OOM;
    if (cudaMalloc((void**)&dsl, sizeof(int) * cap) != cudaSuccess || cudaMalloc((void**)&dst, 16 * (size_t)cap) != cudaSuccess ||
        cudaMallocHost((void**)&hst, 16 * (size_t)cap) != cudaSuccess || cudaMallocHost((void**)&hsl, sizeof(int) * cap) != cudaSuccess) {
        cudaFree(rds);
        if (dsl) cudaFree(dsl);
        if (dst) cudaFree(dst);
        if (hst) cudaFreeHost(hst);
        return RVE_E_OOM;
    }
    if (E.d_rds) {
        CK(cudaMemcpyAsync(rds, E.d_rds, sizeof(Launch) * E.cap, cudaMemcpyDeviceToDevice, E.stream));
        CK(cudaStreamSynchronize(E.stream));
        cudaFree(E.d_rds);
        cudaFree(E.d_slots);
        cudaFree(E.d_status);
        cudaFreeHost(E.h_status);
        cudaFreeHost(E.h_slots);
    }
    E.d_rds = rds;
    E.d_slots = dsl;
    E.d_status = dst;
    E.h_status = hst;
    E.h_slots = hsl;
    for (int s = E.cap; s < cap; ++s) E.free_slots.push_back(s);
    std::sort(E.free_slots.rbegin(), E.free_slots.rend());  // hand out low slots first
    E.mem.resize(cap);
    E.cap = cap;
    for (auto& kv : E.runs) kv.second.dirty = true;  // descriptor array moved
    return RVE_OK;
}

// Whether a member takes the lean local kernel in this run's stage (no lean kernel in the
// plain double stage).
bool member_lean(const rve* h, int stage) {
    if (stage == kStageF64) return false;
    return admm::lean_local(h->L, h->E.exact_local != 0, stage == kStagePolish);
}

int run_upload(Engine& E, BatchRun& r) {
    std::vector<int2> t;
    // local tiles: the members without a lean kernel first (they share one tile launch)
    std::vector<int> local_order;
    for (int pass = 0; pass < 2; ++pass)
        for (int slot : r.active)
            if (member_lean(E.mem[slot].h, r.stage) == (pass == 1)) local_order.push_back(slot);
    for (int c = 0; c < admm::kTileClasses; ++c) {
        t.clear();
        for (int slot : (c == admm::kTilesLocal ? local_order : r.active)) {
            const Launch& L = E.mem[slot].h->L;
            const int cnt = c == admm::kTilesLocal ? admm::tiles_local(L)
                          : c == admm::kTilesX     ? admm::tiles_x(L)
                                                   : admm::tiles_ax(L, c == admm::kTilesAx64);
            for (int j = 0; j < cnt; ++j) t.push_back(make_int2(slot, j));
        }
        if ((int)t.size() > r.cap[c]) {
            if (r.d_tiles[c]) cudaFree(r.d_tiles[c]);
            r.d_tiles[c] = nullptr;
            r.cap[c] = 0;
            if (cudaMalloc((void**)&r.d_tiles[c], std::max<size_t>(t.size(), 1) * sizeof(int2)) != cudaSuccess)
                return RVE_E_OOM;
            r.cap[c] = (int)t.size();
        }
        if (!t.empty())
            CK(cudaMemcpyAsync(r.d_tiles[c], t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, E.stream));
        CK(cudaStreamSynchronize(E.stream));
        r.E.tiles[c] = r.d_tiles[c];
        r.E.ntiles[c] = (int)t.size();
    }
    r.E.stream = E.stream;
    r.E.rds = E.d_rds;
    r.E.rep = &E.mem[r.active.front()].h->L;
    r.E.uniform_n = E.mem[r.active.front()].h->n;
    r.E.uniform_geom = 1;
    r.E.exact_local = 1;
    r.mem.clear();
    r.mem_exact.clear();
    r.mem_tile0.clear();
    int tile0 = 0;
    for (int slot : local_order) {
        if (E.mem[slot].h->n != r.E.uniform_n) r.E.uniform_n = 0;
        const Launch& M = E.mem[slot].h->L;
        const Launch& R0 = E.mem[r.active.front()].h->L;
        if (M.lpb != R0.lpb || M.tk32 != R0.tk32 || M.tk64 != R0.tk64) r.E.uniform_geom = 0;
        if (!E.mem[slot].h->E.exact_local) r.E.exact_local = 0;
        r.mem.push_back(&E.mem[slot].h->L);
        r.mem_exact.push_back((unsigned char)E.mem[slot].h->E.exact_local);
        r.mem_tile0.push_back(tile0);
        tile0 += admm::tiles_local(E.mem[slot].h->L);
    }
    r.E.nmem = (int)r.mem.size();
    r.E.mem = r.mem.data();
    r.E.mem_exact = r.mem_exact.data();
    r.E.mem_tile0 = r.mem_tile0.data();
    for (int f = 0; f < 2; ++f) {
        r.E.smem_x[f] = 0;
        r.E.smem_a[f] = 0;
        for (int slot : r.active) {
            r.E.smem_x[f] = std::max(r.E.smem_x[f], admm::smem_x_bytes(E.mem[slot].h->L, f == 1));
            r.E.smem_a[f] = std::max(r.E.smem_a[f], admm::smem_a_bytes(E.mem[slot].h->L, f == 1));
        }
    }
    if (r.graph) {
        cudaGraphExecDestroy(r.graph);
        r.graph = nullptr;
    }
    r.dirty = false;
    return RVE_OK;
}

int run_chunk(Engine& E, BatchRun& r, int stage) {
    const rve_options& o = E.mem[r.active.front()].h->opt;
    const bool fp64 = stage != kStageF32;
    const bool polish = stage == kStagePolish;
    auto body = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < o.check_every && e == cudaSuccess; ++i) {
            e = polish ? admm::launch_fft_incr(r.E) : admm::launch_fft(r.E, fp64);
            if (e == cudaSuccess) e = admm::launch_local(r.E, fp64, false, false, polish ? 2 : 0);
            if (e == cudaSuccess && o.rho_policy == RVE_RHO_ADAPTIVE) e = admm::launch_local(r.E, fp64, true, true);
        }
        return e;
    };
    if (!o.use_graph) return body() == cudaSuccess ? RVE_OK : RVE_E_CUDA;
    if (!r.graph) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(E.stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = body();
        const cudaError_t e2 = cudaStreamEndCapture(E.stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return RVE_E_CUDA;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&r.graph, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return RVE_E_CUDA;
    }
    CK(cudaGraphLaunch(r.graph, E.stream));
    return RVE_OK;
}

void run_insert(Engine& E, int slot) {
    const Member& m = E.mem[slot];
    BatchRun& r = E.runs[RunKey(m.h->dim, m.h->L.model, m.stage, size_class(m.h))];
    r.stage = m.stage;
    r.active.insert(std::lower_bound(r.active.begin(), r.active.end(), slot), slot);
    r.dirty = true;
}

void run_remove(Engine& E, int slot) {
    const Member& m = E.mem[slot];
    auto it = E.runs.find(RunKey(m.h->dim, m.h->L.model, m.stage, size_class(m.h)));
    if (it == E.runs.end()) return;
    auto pos = std::find(it->second.active.begin(), it->second.active.end(), slot);
    if (pos != it->second.active.end()) {
        it->second.active.erase(pos);
        it->second.dirty = true;
    }
}

// Start a solve of h in the engine; returns the slot (>= 0) or an error.
int engine_add(Engine& E, rve* h, const double Fbar[9], double rho, double tol) {
    int rc = check_solve_args(h, Fbar, rho, tol);
    if (rc) return rc;
    if (E.free_slots.empty() && (rc = engine_reserve(E, E.cap + 1))) return rc;
    const int slot = E.free_slots.back();
    E.free_slots.pop_back();
    h->launches = 0;
    rc = begin_solve(h, Fbar, rho, tol, E.stream);
    if (rc) {
        E.free_slots.push_back(slot);
        return rc;
    }
    CK(cudaMemcpyAsync(E.d_rds + slot, &h->L, sizeof(Launch), cudaMemcpyHostToDevice, E.stream));
    Member& m = E.mem[slot];
    m.h = h;
    m.k0 = h->hctrl->k;
    m.ksw = -1;
    m.stage = h->opt.precision == RVE_FP64 ? kStageF64 : kStageF32;
    m.running = h->hctrl->done == admm::kRunning;
    if (m.running) {
        admm::Exec Ei = h->E;  // the member's own tile tables for its first local step
        Ei.stream = E.stream;
        if (admm::launch_local(Ei, m.stage != kStageF32, true, false) != cudaSuccess) return RVE_E_CUDA;
        h->launches += 1;
        run_insert(E, slot);
    }
    return slot;
}

int engine_running(const Engine& E) {
    int n = 0;
    for (int s = 0; s < E.cap; ++s) n += (E.mem[s].h && E.mem[s].running) ? 1 : 0;
    return n;
}

// One chunk of every run; returns the slots that finished in this tick.
int engine_tick(Engine& E, std::vector<int>& finished) {
    finished.clear();
    int nrun = 0;
    for (auto& kv : E.runs) {
        BatchRun& r = kv.second;
        if (r.active.empty()) continue;
        if (r.dirty) {
            const int rc = run_upload(E, r);
            if (rc) return rc;
        }
        const int rc = run_chunk(E, r, std::get<2>(kv.first));
        if (rc) return rc;
        const rve* h0 = E.mem[r.active.front()].h;
        const int per = admm::fft_stages(h0->dim) + 1 + (h0->opt.rho_policy == RVE_RHO_ADAPTIVE ? 1 : 0);
        for (int slot : r.active) E.mem[slot].h->launches += (long long)h0->opt.check_every * per;
        nrun += (int)r.active.size();
    }
    if (nrun == 0) return RVE_OK;
    int cnt = 0;
    for (int s = 0; s < E.cap; ++s)
        if (E.mem[s].h && E.mem[s].running) E.h_slots[cnt++] = s;
    CK(cudaMemcpyAsync(E.d_slots, E.h_slots, sizeof(int) * cnt, cudaMemcpyHostToDevice, E.stream));
    k_gather_status<<<(cnt + 127) / 128, 128, 0, E.stream>>>(E.d_rds, E.d_slots, cnt, E.d_status);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(E.h_status, E.d_status, 16 * (size_t)cnt, cudaMemcpyDeviceToHost, E.stream));
    CK(cudaStreamSynchronize(E.stream));
    std::vector<int> slots(E.h_slots, E.h_slots + cnt);
    std::vector<long long> st(E.h_status, E.h_status + 2 * cnt);
    for (int i = 0; i < cnt; ++i) {
        if (st[2 * i] == admm::kRunning) continue;
        const int slot = slots[i];
        Member& m = E.mem[slot];
        rve* h = m.h;
        run_remove(E, slot);
        if (read_ctrl_on(h, E.stream)) return RVE_E_CUDA;
        if (h->opt.precision == RVE_MIXED && m.stage == kStageF32 && h->hctrl->done == admm::kSwitch) {
            m.ksw = h->hctrl->k;
            const bool direct = switch_direct_ok(h);
            if (switch_to_double(h, E.stream, direct)) return RVE_E_CUDA;
            if (!direct) {
                // the member's first double iterations (local step, one full double
                // projection, local step writing R) run on its own tile tables
                admm::Exec Ei = h->E;
                Ei.stream = E.stream;
                if (admm::launch_local(Ei, true, true, false) != cudaSuccess) return RVE_E_CUDA;
                if (admm::launch_fft(Ei, true) != cudaSuccess) return RVE_E_CUDA;
                if (admm::launch_local(Ei, true, false, false, 1) != cudaSuccess) return RVE_E_CUDA;
                if (admm::launch_polish_state(h->L, true, E.stream) != cudaSuccess) return RVE_E_CUDA;
                h->launches += admm::fft_stages(h->dim) + 4;
            }
            m.stage = kStagePolish;
            run_insert(E, slot);
        } else {
            m.running = false;
            finished.push_back(slot);
        }
    }
    return RVE_OK;
}

// Info of a finished member and release of its slot.
void engine_release(Engine& E, int slot, double ms, rve_solve_info* info) {
    Member& m = E.mem[slot];
    rve* h = m.h;
    if (m.stage == kStagePolish) {  // back to the double state (no-op unless it was converted),
        admm::launch_polish_state(h->L, false, E.stream);  // finished before the handle's own
        cudaStreamSynchronize(E.stream);                   // stream reads it
        h->launches += 2;
    }
    int fp64_iters = 0;
    if (h->opt.precision == RVE_FP64)
        fp64_iters = (int)(h->hctrl->k - m.k0);
    else if (m.ksw >= 0)
        fp64_iters = (int)(h->hctrl->k - m.ksw);
    fill_info(h, m.k0, fp64_iters, ms, info);
    if (m.running) run_remove(E, slot);
    m = Member();
    E.free_slots.push_back(slot);
}

}  // namespace

struct rve_batch {
    std::vector<rve*> m;
    cudaStream_t user_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev0 = nullptr, ev1 = nullptr;
    Engine E;
};

extern "C" {

int rve_batch_create(rve_batch_t* out, rve_t* handles, int count, void* cuda_stream) {
    if (!out || !handles || count < 1) return RVE_E_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!handles[i]) return RVE_E_INVALID_ARG;
        if (!handles[i]->material_set) return RVE_E_STATE;
        if (handles[i]->opt.precision != handles[0]->opt.precision ||
            handles[i]->opt.rho_policy != handles[0]->opt.rho_policy)
            return RVE_E_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return RVE_E_INVALID_ARG;
    }
    rve_batch* b = new (std::nothrow) rve_batch();
    if (!b) return RVE_E_OOM;
    auto fail = [&](int code) {
        rve_batch_destroy(b);
        return code;
    };
    b->m.assign(handles, handles + count);
    b->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&b->E.stream, cudaStreamNonBlocking) != cudaSuccess) return fail(RVE_E_CUDA);
    if (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(RVE_E_CUDA);
    if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) return fail(RVE_E_CUDA);
    const int rc = engine_reserve(b->E, count);
    if (rc) return fail(rc);
    *out = b;
    return RVE_OK;
}

void rve_batch_destroy(rve_batch_t b) {
    if (!b) return;
    engine_free(b->E);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->E.stream) cudaStreamDestroy(b->E.stream);
    delete b;
}

int rve_batch_solve(rve_batch_t b, const double* Fbars, const double* rhos, double tol, rve_solve_info* infos) {
    if (!b || !Fbars || !rhos) return RVE_E_INVALID_ARG;
    const int count = (int)b->m.size();
    for (int i = 0; i < count; ++i) {
        const int rc = check_solve_args(b->m[i], Fbars + 9 * i, rhos[i], tol);
        if (rc) return rc;
    }
    Engine& E = b->E;
    CK(cudaEventRecord(b->ev_in, b->user_stream));
    CK(cudaStreamWaitEvent(E.stream, b->ev_in, 0));
    CK(cudaEventRecord(b->ev0, E.stream));
    std::vector<int> slot(count);
    for (int i = 0; i < count; ++i) {
        slot[i] = engine_add(E, b->m[i], Fbars + 9 * i, rhos[i], tol);
        if (slot[i] < 0) return slot[i];
    }
    std::vector<int> finished;
    while (engine_running(E) > 0) {
        const int rc = engine_tick(E, finished);
        if (rc) return rc;
    }
    CK(cudaEventRecord(b->ev1, E.stream));
    CK(cudaEventSynchronize(b->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    int status = RVE_OK;
    for (int i = 0; i < count; ++i) {
        rve* h = b->m[i];
        if (read_ctrl_on(h, E.stream)) return RVE_E_CUDA;
        engine_release(E, slot[i], ms, infos ? infos + i : nullptr);
        const int st = status_of(h->hctrl->done);
        if (status == RVE_OK && st != RVE_OK) status = st;
    }
    return status;
}

}  // extern "C"

// ================================================================== server (continuous batching)

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long ticket = 0;
    int dim = 3, n = 0, model = 0, nphase = 0, nparam = 0;
    std::vector<uint8_t> phase;
    std::vector<double> params, n0;
    double Fbar[9] = {};
    double rho = 10.0, tol = 1e-8;
    size_t bytes = 0;
    double t_submit = 0.0, t_admit = 0.0;
};

struct Finished {
    int status = RVE_OK;
    double S[9] = {};
    rve_solve_info info{};
    double queue_ms = 0.0, latency_ms = 0.0;
};

using ShapeKey = std::tuple<int, int, int>;

}  // namespace

struct rve_server {
    rve_options opt{};
    size_t budget = 0, used = 0;  // bytes of workspaces held (active + pooled)
    cudaStream_t user_stream = nullptr;
    Engine E;
    std::deque<Request> queue;
    std::map<int, Request> active;  // slot -> request (inputs dropped)
    std::map<int, rve*> active_h;
    std::map<long long, Finished> done;
    std::multimap<ShapeKey, rve*> pool;  // idle handles by (dim, n, model)
    long long next_ticket = 1;
    long long completed = 0;
};

namespace {

size_t server_bytes(const rve_server* s, int dim, int n, int model) {
    return layout(dim, n, model, s->opt.precision, s->opt.max_iter).total;
}

void server_drop_pool(rve_server* s, size_t need) {
    while (s->used + need > s->budget && !s->pool.empty()) {
        auto it = s->pool.begin();
        rve* h = it->second;
        s->used -= server_bytes(s, h->dim, h->n, h->model);
        rve_destroy(h);
        s->pool.erase(it);
    }
}

// Admit queued requests in arrival order while their workspaces fit the budget.
// A request whose material or load the library rejects when it is admitted ends
// by itself with that status (NaN stress); the other requests and later steps are
// unaffected.
void server_reject(rve_server* s, const Request& r, int status) {
    Finished f;
    f.status = status;
    for (int i = 0; i < 9; ++i) f.S[i] = NAN;
    f.info.status = status;
    const double t = now_ms();
    f.queue_ms = t - r.t_submit;
    f.latency_ms = t - r.t_submit;
    s->done[r.ticket] = f;
    s->completed += 1;
}

int server_admit(rve_server* s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request& r = *it;
        const ShapeKey key(r.dim, r.n, r.model);
        rve* h = nullptr;
        auto pit = s->pool.find(key);
        if (pit != s->pool.end()) {
            h = pit->second;
            s->pool.erase(pit);
        } else {
            server_drop_pool(s, r.bytes);
            if (s->used + r.bytes > s->budget) {
                ++it;
                continue;
            }
            const int rc = rve_create(&h, r.dim, r.n, r.model, &s->opt, s->user_stream);
            if (rc == RVE_E_OOM) {
                ++it;
                continue;
            }
            if (rc) return rc;
            s->used += r.bytes;
        }
        int rc = rve_set_material(h, r.phase.data(), r.nphase, r.params.data(), r.nparam,
                                  r.model == RVE_LCE ? r.n0.data() : nullptr);
        if (rc) {
            rve_destroy(h);
            s->used -= r.bytes;
            if (rc != RVE_E_INVALID_ARG) return rc;
            server_reject(s, r, rc);
            it = s->queue.erase(it);
            continue;
        }
        const int slot = engine_add(s->E, h, r.Fbar, r.rho, r.tol);
        if (slot < 0) {
            rve_destroy(h);
            s->used -= r.bytes;
            if (slot != RVE_E_INVALID_ARG) return slot;
            server_reject(s, r, slot);
            it = s->queue.erase(it);
            continue;
        }
        r.t_admit = now_ms();
        r.phase.clear();
        r.phase.shrink_to_fit();
        r.params.clear();
        r.n0.clear();
        r.n0.shrink_to_fit();
        s->active[slot] = std::move(r);
        s->active_h[slot] = h;
        it = s->queue.erase(it);
    }
    return RVE_OK;
}

int server_retire(rve_server* s, int slot) {
    rve* h = s->active_h[slot];
    Request& r = s->active[slot];
    Finished f;
    if (read_ctrl_on(h, s->E.stream)) return RVE_E_CUDA;
    f.status = status_of(h->hctrl->done);
    engine_release(s->E, slot, 0.0, &f.info);
    const int rc = rve_stress(h, f.S);
    if (rc) return rc;
    const double t = now_ms();
    f.queue_ms = r.t_admit - r.t_submit;
    f.latency_ms = t - r.t_submit;
    f.info.time_ms = t - r.t_admit;
    s->done[r.ticket] = f;
    s->pool.insert({ShapeKey(h->dim, h->n, h->model), h});
    s->active.erase(slot);
    s->active_h.erase(slot);
    s->completed += 1;
    return RVE_OK;
}

}  // namespace

extern "C" {

int rve_server_create(rve_server_t* out, size_t mem_budget_bytes, const rve_options* opt, void* cuda_stream) {
    if (!out || mem_budget_bytes == 0) return RVE_E_INVALID_ARG;
    *out = nullptr;
    rve_options o;
    rve_default_options(&o);
    if (opt) o = *opt;
    if (check_options(o)) return RVE_E_INVALID_ARG;
    rve_server* s = new (std::nothrow) rve_server();
    if (!s) return RVE_E_OOM;
    s->opt = o;
    s->budget = mem_budget_bytes;
    s->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&s->E.stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return RVE_E_CUDA;
    }
    *out = s;
    return RVE_OK;
}

void rve_server_destroy(rve_server_t s) {
    if (!s) return;
    engine_free(s->E);
    for (auto& kv : s->active_h) rve_destroy(kv.second);
    for (auto& kv : s->pool) rve_destroy(kv.second);
    if (s->E.stream) cudaStreamDestroy(s->E.stream);
    delete s;
}

int rve_server_submit(rve_server_t s, int dim, int n, int model, const uint8_t* phase, int nphase,
                      const double* params, int nparam, const double* n0, const double Fbar[9], double rho,
                      double tol, long long* ticket) {
    if (!s || !phase || !params || !Fbar || !ticket) return RVE_E_INVALID_ARG;
    if ((dim != 2 && dim != 3) || !valid_n(n)) return RVE_E_INVALID_ARG;
    if (model != RVE_NEOHOOKE && model != RVE_LINEAR && model != RVE_LCE) return RVE_E_INVALID_ARG;
    if (model == RVE_LCE && (dim != 3 || !n0 || nparam < 5)) return RVE_E_INVALID_ARG;
    if (nphase < 1 || nphase > 256 || nparam < 2 || nparam > admm::kMaxParam) return RVE_E_INVALID_ARG;
    if (!(rho > 0) || !isfinite(rho) || isnan(tol)) return RVE_E_INVALID_ARG;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(Fbar[i])) return RVE_E_INVALID_ARG;
    const double det2 = Fbar[0] * Fbar[4] - Fbar[1] * Fbar[3];
    const double det3 = Fbar[0] * (Fbar[4] * Fbar[8] - Fbar[5] * Fbar[7]) -
                        Fbar[1] * (Fbar[3] * Fbar[8] - Fbar[5] * Fbar[6]) +
                        Fbar[2] * (Fbar[3] * Fbar[7] - Fbar[4] * Fbar[6]);
    if (!((dim == 2 ? det2 : det3) > 0)) return RVE_E_INVALID_ARG;  // as rve_solve
    const long long V = dim == 3 ? (long long)n * n * n : (long long)n * n;
    for (long long v = 0; v < V; ++v)
        if (phase[v] >= nphase) return RVE_E_INVALID_ARG;
    const size_t bytes = server_bytes(s, dim, n, model);
    if (bytes > s->budget) return RVE_E_OOM;  // can never be admitted
    Request r;
    r.ticket = s->next_ticket++;
    r.dim = dim;
    r.n = n;
    r.model = model;
    r.nphase = nphase;
    r.nparam = nparam;
    r.phase.assign(phase, phase + V);
    r.params.assign(params, params + (size_t)nphase * nparam);
    if (model == RVE_LCE) r.n0.assign(n0, n0 + 3 * V);
    for (int i = 0; i < 9; ++i) r.Fbar[i] = Fbar[i];
    r.rho = rho;
    r.tol = tol;
    r.bytes = bytes;
    r.t_submit = now_ms();
    *ticket = r.ticket;
    s->queue.push_back(std::move(r));
    return RVE_OK;
}

int rve_server_step(rve_server_t s, int* active_out, int* queued_out) {
    if (!s) return RVE_E_INVALID_ARG;
    int rc = server_admit(s);
    if (rc) return rc;
    if (engine_running(s->E) > 0) {
        std::vector<int> finished;
        rc = engine_tick(s->E, finished);
        if (rc) return rc;
        for (int slot : finished) {
            rc = server_retire(s, slot);
            if (rc) return rc;
        }
    }
    if (active_out) *active_out = (int)s->active.size();
    if (queued_out) *queued_out = (int)s->queue.size();
    return RVE_OK;
}

int rve_server_poll(rve_server_t s, long long ticket, double S[9], rve_solve_info* info, double* latency_ms,
                    double* queue_ms) {
    if (!s) return RVE_E_INVALID_ARG;
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        for (const Request& r : s->queue)
            if (r.ticket == ticket) return RVE_E_BUSY;
        for (const auto& kv : s->active)
            if (kv.second.ticket == ticket) return RVE_E_BUSY;
        return RVE_E_NOT_FOUND;
    }
    const Finished& f = it->second;
    if (S)
        for (int i = 0; i < 9; ++i) S[i] = f.S[i];
    if (info) *info = f.info;
    if (latency_ms) *latency_ms = f.latency_ms;
    if (queue_ms) *queue_ms = f.queue_ms;
    const int st = f.status;
    s->done.erase(it);
    return st == RVE_OK ? RVE_OK : st;
}

int rve_server_cancel(rve_server_t s, long long ticket) {
    if (!s) return RVE_E_INVALID_ARG;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->ticket == ticket) {
            s->queue.erase(it);
            return RVE_OK;
        }
    for (auto& kv : s->active)
        if (kv.second.ticket == ticket) {
            const int slot = kv.first;
            rve* h = s->active_h[slot];
            CK(cudaStreamSynchronize(s->E.stream));
            engine_release(s->E, slot, 0.0, nullptr);
            s->pool.insert({ShapeKey(h->dim, h->n, h->model), h});
            s->active.erase(slot);
            s->active_h.erase(slot);
            return RVE_OK;
        }
    return RVE_E_NOT_FOUND;
}

int rve_server_stats(rve_server_t s, long long* queued, long long* active, long long* completed, size_t* bytes_used) {
    if (!s) return RVE_E_INVALID_ARG;
    if (queued) *queued = (long long)s->queue.size();
    if (active) *active = (long long)s->active.size();
    if (completed) *completed = s->completed;
    if (bytes_used) *bytes_used = s->used;
    return RVE_OK;
}

}  // extern "C"

// ================================================================== FFT autotuner

namespace {

// distinct orderings of a radix multiset
std::vector<std::vector<int>> radix_orders(int L) {
    int rad[admm::kMaxPasses];
    const int np = admm::factor_radices(L, rad);
    std::vector<int> v(rad, rad + np);
    std::sort(v.begin(), v.end());
    std::vector<std::vector<int>> out;
    do out.push_back(v);
    while (std::next_permutation(v.begin(), v.end()) && out.size() < 12);
    return out;
}

int upload_tiles_tmp(rve* h, const Launch& L, int2** buf, int* cap, int cls, admm::Exec& E) {
    const int cnt = cls == admm::kTilesX ? admm::tiles_x(L) : admm::tiles_ax(L, cls == admm::kTilesAx64);
    if (cnt > *cap) {
        if (*buf) cudaFree(*buf);
        *buf = nullptr;
        if (cudaMalloc((void**)buf, sizeof(int2) * cnt) != cudaSuccess) return RVE_E_OOM;
        *cap = cnt;
    }
    std::vector<int2> t(cnt);
    for (int i = 0; i < cnt; ++i) t[i] = make_int2(0, i);
    CK(cudaMemcpyAsync(*buf, t.data(), sizeof(int2) * cnt, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    E.tiles[cls] = *buf;
    E.ntiles[cls] = cnt;
    return RVE_OK;
}

// min over reps of the summed device time of the chosen FFT stages
int time_stages(rve* h, admm::Exec& E, bool fp64, const std::vector<int>& stages, double* best) {
    const int S = admm::fft_stages(h->dim);
    std::vector<cudaEvent_t> ev(S + 1);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    *best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(ev[0], h->stream));
        for (int st = 0; st < S; ++st) {
            if (admm::launch_fft(E, fp64, st) != cudaSuccess) return RVE_E_CUDA;
            CK(cudaEventRecord(ev[st + 1], h->stream));
        }
        CK(cudaEventSynchronize(ev[S]));
        double t = 0.0;
        for (int st : stages) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[st], ev[st + 1]);
            t += ms;
        }
        if (rep > 0) *best = std::min(*best, t);  // first repetition warms up
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return RVE_OK;
}

}  // namespace

extern "C" {

int rve_autotune(int dim, int n, int precision, const char* cache_path, double* best_ms) {
    if ((dim != 2 && dim != 3) || !valid_n(n) || precision < RVE_FP64 || precision > RVE_FP32)
        return RVE_E_INVALID_ARG;
    const bool fp64 = precision == RVE_FP64;
    rve_options o;
    rve_default_options(&o);
    o.precision = fp64 ? RVE_FP64 : RVE_FP32;
    o.max_iter = 1;
    rve* h = nullptr;
    int rc = rve_create(&h, dim, n, RVE_NEOHOOKE, &o, nullptr);
    if (rc) return rc;
    const long long V = h->V;
    std::vector<uint8_t> ph((size_t)V, 0);
    const double par[2] = {1.0, 1.5};
    const double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int2 *tx = nullptr, *ta = nullptr;
    int capx = 0, capa = 0;
    admm::Geometry best_g = admm::default_geometry(dim, n);
    double best_x = 1e30, best_a = 1e30;
    auto cleanup = [&](int code) {
        if (tx) cudaFree(tx);
        if (ta) cudaFree(ta);
        rve_destroy(h);
        return code;
    };
    if ((rc = rve_set_material(h, ph.data(), 1, par, 2, nullptr))) return cleanup(rc);
    if ((rc = begin_solve(h, I, 10.0, -1.0, h->stream))) return cleanup(rc);
    const int H = n / 2, nlines = dim == 3 ? n * n : n;
    const int S = admm::fft_stages(dim);
    const std::vector<int> xstages = {0, S - 1};
    std::vector<int> astages;
    for (int st = 1; st < S - 1; ++st) astages.push_back(st);
    const auto half_orders = radix_orders(H);
    const auto full_orders = radix_orders(n);
    std::vector<int> lpbs;
    for (int t : {32, 128, 512, 1024, 2048, 4096, 8192}) {
        const int l = std::max(1, std::min(nlines, t / n));
        if (std::find(lpbs.begin(), lpbs.end(), l) == lpbs.end()) lpbs.push_back(l);
    }
    std::vector<int> tks;
    for (int t : {1, 2, 4, 8, 16, 32})
        if (t <= H) tks.push_back(t);
    if (tks.empty()) tks.push_back(H);
    admm::Exec E = h->E;
    const int acls = fp64 ? admm::kTilesAx64 : admm::kTilesAx32;
    for (int pass = 0; pass < 2; ++pass) {
        const bool xpass = pass == 0;
        const size_t nc = xpass ? lpbs.size() * half_orders.size() : tks.size() * full_orders.size();
        for (size_t c = 0; c < nc; ++c) {
            admm::Geometry g = best_g;
            if (xpass) {
                g.lpb = lpbs[c / half_orders.size()];
                const auto& ord = half_orders[c % half_orders.size()];
                g.np_half = (int)ord.size();
                for (size_t i = 0; i < ord.size(); ++i) g.rad_half[i] = ord[i];
            } else {
                (fp64 ? g.tk64 : g.tk32) = tks[c / full_orders.size()];
                const auto& ord = full_orders[c % full_orders.size()];
                g.np_full = (int)ord.size();
                for (size_t i = 0; i < ord.size(); ++i) g.rad_full[i] = ord[i];
            }
            admm::apply_geometry(h->L, g);
            if ((rc = write_desc(h))) return cleanup(rc);
            if ((rc = upload_tiles_tmp(h, h->L, &tx, &capx, admm::kTilesX, E))) return cleanup(rc);
            if ((rc = upload_tiles_tmp(h, h->L, &ta, &capa, acls, E))) return cleanup(rc);
            for (int f = 0; f < 2; ++f) {
                E.smem_x[f] = admm::smem_x_bytes(h->L, f == 1);
                E.smem_a[f] = admm::smem_a_bytes(h->L, f == 1);
            }
            if (E.smem_x[fp64] > 200 * 1024 || E.smem_a[fp64] > 200 * 1024) continue;
            double t = 0.0;
            if ((rc = time_stages(h, E, fp64, xpass ? xstages : astages, &t))) return cleanup(rc);
            if (xpass && t < best_x) {
                best_x = t;
                best_g.lpb = g.lpb;
                best_g.np_half = g.np_half;
                for (int i = 0; i < admm::kMaxPasses; ++i) best_g.rad_half[i] = g.rad_half[i];
            } else if (!xpass && t < best_a) {
                best_a = t;
                (fp64 ? best_g.tk64 : best_g.tk32) = fp64 ? g.tk64 : g.tk32;
                best_g.np_full = g.np_full;
                for (int i = 0; i < admm::kMaxPasses; ++i) best_g.rad_full[i] = g.rad_full[i];
            }
        }
        (void)nlines;
    }
    admm::register_geometry(dim, n, best_g);
    if (best_ms) *best_ms = best_x + best_a;
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {  // one JSON object per line
            fprintf(f, "{\"kind\": \"rve-fft-geometry\", \"dim\": %d, \"n\": %d, \"precision\": %d, \"lpb\": %d, "
                       "\"tk64\": %d, \"tk32\": %d, \"rad_half\": [",
                    dim, n, precision, best_g.lpb, best_g.tk64, best_g.tk32);
            for (int i = 0; i < best_g.np_half; ++i) fprintf(f, "%s%d", i ? ", " : "", best_g.rad_half[i]);
            fprintf(f, "], \"rad_full\": [");
            for (int i = 0; i < best_g.np_full; ++i) fprintf(f, "%s%d", i ? ", " : "", best_g.rad_full[i]);
            fprintf(f, "], \"ms\": %.6f}\n", best_x + best_a);
            fclose(f);
        }
    }
    return cleanup(RVE_OK);
}

// Cache lines: {"kind": "rve-fft-geometry", "dim": .., "n": .., "precision": .., "lpb": ..,
// "tk64": .., "tk32": .., "rad_half": [..], "rad_full": [..], "ms": ..} -- the fields this
// writer emits, read back by key (not a general JSON parser).
namespace {
const char* json_key(const char* line, const char* key) {
    char pat[32];
    snprintf(pat, sizeof pat, "\"%s\"", key);
    const char* p = strstr(line, pat);
    if (!p) return nullptr;
    p += strlen(pat);
    while (*p == ' ') ++p;
    if (*p != ':') return nullptr;
    ++p;
    while (*p == ' ') ++p;
    return p;
}
bool json_int(const char* line, const char* key, int* out) {
    const char* p = json_key(line, key);
    if (!p) return false;
    char* e = nullptr;
    const long v = strtol(p, &e, 10);
    if (e == p || v < INT32_MIN || v > INT32_MAX) return false;
    *out = (int)v;
    return true;
}
// a list of radices (2, 3, 4 or 8) whose product is want; count in *np
bool json_radices(const char* line, const char* key, int* rad, int* np, int want) {
    const char* p = json_key(line, key);
    if (!p || *p != '[') return false;
    ++p;
    int cnt = 0, prod = 1;
    for (;;) {
        while (*p == ' ') ++p;
        if (*p == ']') break;
        char* e = nullptr;
        const long r = strtol(p, &e, 10);
        if (e == p || !(r == 2 || r == 3 || r == 4 || r == 8) || cnt >= admm::kMaxPasses) return false;
        rad[cnt++] = (int)r;
        prod *= (int)r;
        p = e;
        while (*p == ' ') ++p;
        if (*p == ',') ++p;
        else if (*p != ']') return false;
    }
    *np = cnt;
    return cnt > 0 && prod == want;
}
}  // namespace

int rve_autotune_load(const char* cache_path) {
    if (!cache_path) return RVE_E_INVALID_ARG;
    FILE* f = fopen(cache_path, "r");
    if (!f) return RVE_E_NOT_FOUND;
    char line[1024];
    int loaded = 0;
    while (fgets(line, sizeof line, f)) {
        admm::Geometry g{};
        int dim = 0, n = 0, prec = 0;
        bool ok = strstr(line, "\"rve-fft-geometry\"") != nullptr && json_int(line, "dim", &dim) &&
                  json_int(line, "n", &n) && json_int(line, "precision", &prec) && json_int(line, "lpb", &g.lpb) &&
                  json_int(line, "tk64", &g.tk64) && json_int(line, "tk32", &g.tk32);
        ok = ok && (dim == 2 || dim == 3) && valid_n(n);
        ok = ok && json_radices(line, "rad_half", g.rad_half, &g.np_half, n / 2) &&
             json_radices(line, "rad_full", g.rad_full, &g.np_full, n);
        ok = ok && g.lpb >= 1 && g.tk64 >= 1 && g.tk64 <= n / 2 && g.tk32 >= 1 && g.tk32 <= n / 2;
        if (ok) {
            admm::register_geometry(dim, n, g);
            ++loaded;
        }
    }
    fclose(f);
    return loaded;
}

}  // extern "C"
