// Internal definitions shared by the solver's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace admm {

constexpr int kMaxPasses = 16;
constexpr int kLocalThreads = 128;    // threads per block of the local-step kernels
constexpr int kLocalTileCap = 152 * 12;  // local tiles of one RVE at most (whole waves at 2, 3, 4 or 6
                                         // resident blocks per SM)
constexpr int kFftThreads = 256;      // threads per block of the FFT kernels
// per-phase material constants: the law's own (mu, lam first); the LCE adds r, alpha,
// kappa_F (2-4), the derived a, c1, c2 (5-7), the dissipation weights nu_F/dt, nu_n/dt
// (8, 9) and the incompressibility flag (10)
constexpr int kMaxParam = 12;
constexpr int kPartialStride = 20;
// fraction-converged local steps: counts of voxels whose Newton met its test within
// 2, 4, ..., 2 kNewtonBins iterations
constexpr int kNewtonBins = 16;
// residual history entry per iteration: r_p, r_d, rho of the check, then r_l of the
// local step fused into the same pass (the next iteration's Step 1)
constexpr int kHistStride = 4;    // doubles per block in the partial-sum buffer

enum Done : int { kRunning = 0, kConverged = 1, kCapped = 2, kNumerical = 3, kSwitch = 4 };
// kLceInc: the LCE with the incompressible network, chosen by the material table
// (the public model stays RVE_LCE)
enum Model : int { kNeoHooke = 0, kLinear = 1, kLce = 2, kLceInc = 3 };
__host__ __device__ constexpr bool is_lce(int m) { return m == kLce || m == kLceInc; }

// Per-RVE control block in device memory.  Every kernel reads it at entry (the
// ping-pong parity, the penalty, the stop flag); only the last block of the
// fused local kernel and the host write it.  Field order is part of the
// host/device contract within this library only.
struct Ctrl {
    double Fbar[9];      // macroscopic gradient (row-major, 3x3; d x d block used)
    double rho;          // penalty of the current iteration
    double inv_rho;
    double mu_ref;       // modulus in r_d
    double tol;
    double rho_kappa, rho_tau, rho_min;
    double switch_tol;   // float phase of mixed mode: promote once max(r_p, r_d) <= this
    double best;         // best max(r_p, r_d) of the float phase (stagnation test)
    double r_p, r_d;     // residuals of the last completed iteration
    double local_ratio;  // f > 0: inexact local steps, |grad phi| <= f mu_ref r_d per voxel
    double local_fraction; // p > 0: Newton capped where a fraction p of voxels converged
    int newton_cap_max;  // the configured per-voxel Newton cap
    unsigned int newton_hist[kNewtonBins];  // this pass's converged-voxel counts (zeroed by the last block)
    double rd_local;     // r_d of the check before the last one (the redone local step's)
    double r_l;          // local residual of the last fused pass's local step (f > 0 only)
    double Fbar_prev[9]; // <F> of the previous iteration (r_d under mixed control)
    unsigned free_mask;  // mixed control: bit 3i+j set = <F_ij> free, <S_ij> -> 0
    int dw_state;        // 1 while F and Lambda are held as double-words (polish)
    int div_given;       // 1: the next increment x-forward pass transforms the divergence
                         // already in D32 (the switch's residual) instead of D^T R
    int z_valid;         // polish: 1 once the linearisation offsets Z (double Lambda buffer) are formed
    // r_d from the spectral solve (Launch::Sprev): spec_have = Sprev holds u^_k when the
    // z pass of iteration k starts; spec_next = that pass stored u^_{k+1}; spec_sum = that
    // pass wrote its tiles' sums of |k|^2 |u^_{k+1} - u^_k|^2 (read by the local pass)
    int spec_have, spec_next, spec_sum;
    // polish entered by the direct switch: u~ as float pairs (high parts fixed at the
    // switch, in both double u~ buffers; low parts accumulate the increments), u~_k's pair
    // in buffer (k + 1) & 1, converted back to double at the polish's end
    int u_pair;
    double stress[9];    // <W_F(F)> of the current state (written by the stress kernel)
    double lam_mean[9];  // <Lambda>
    long long k;         // iterations completed over the handle's life: F_k, u~_k live in buffer k & 1
    long long k_start;   // value of k when the running solve began
    long long k_cap;     // solve stops when k reaches this
    int done;            // enum Done
    int adaptive;        // eq. rho-update on
    int phase_fp32;      // 1 while a float phase of RVE_MIXED runs (switch rules on)
    int stall;           // float-phase iterations without a 10 % improvement of best
    int rho_changed;     // last iteration changed rho: the speculative local step is redone
    int newton_cap;
    double newton_tol;
    int newton_max;      // largest per-voxel Newton count of the last fused pass
    int hist_cap;        // capacity of the residual history (entries)
    unsigned long long newton_fail;
    unsigned int counter; // last-block counter of the fused local kernel
    unsigned int counter2;// last-block counter of the stress kernel
};

// Division by a divisor d >= 1 fixed at plan time, for dividends below 2^31:
// floor(q / d) = (2q * m) >> (32 + l) with l = ceil(log2 d) and the rounded-up
// reciprocal m = ceil(2^(31+l) / d) < 2^32 (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994).  With m d = 2^(31+l) + e,
// 0 <= e < d <= 2^l, the product overshoots q / d by q e / (d 2^(31+l)) < 1 / d,
// which never reaches the next integer.  One multiply-high and two shifts
// instead of the integer divide sequence.
struct FastDiv {
    unsigned d, m, l;
};
inline FastDiv make_fastdiv(unsigned d) {
    unsigned l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long num = 1ull << (31 + l);
    return FastDiv{d, (unsigned)((num + d - 1) / d), l};
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned q, const FastDiv& f) { return __umulhi(q << 1, f.m) >> f.l; }
#endif

// One Stockham pass: butterflies per transform nb = L / R, span Ns of the radices
// already applied, and the twiddle stride N / (Ns R) into the table exp(-2 pi i m / N).
struct FftPass {
    FastDiv nb, ns;
    int tstep;
};

// Stockham plan for one grid size: radix sequences for the half-length x
// transform (N/2) and the full-length y/z transforms (N), with the divisors the
// kernels' index arithmetic needs.
struct FftPlan {
    int n;
    int np_half, np_full;
    int rad_half[kMaxPasses];
    int rad_full[kMaxPasses];
    FftPass pass_half[kMaxPasses];
    FftPass pass_full[kMaxPasses];
    FastDiv div_n, div_h;      // N, N/2
    FastDiv div_tk64, div_tk32; // y/z tile widths
};

// Everything the kernels need about one RVE.  A copy lives in device memory (the
// per-RVE descriptor read by the tile-loop kernels); pointers of the precision not
// in use may be null.
struct Launch {
    cudaStream_t stream;
    int dim, n, model;
    long long V;
    int local_blocks;      // blocks (tiles) of the local kernel for this RVE
    int local_chunk;       // voxels one local tile covers per sweep (<= kLocalThreads)
    int lpb, xblocks;      // x passes: lines per block, blocks
    int tk64, tk32;        // y/z passes: columns per tile (double / float)
    Ctrl* ctrl;
    double* hist;          // 3 doubles per iteration: r_p, r_d, rho
    double* partials;      // kPartialStride doubles per local block
    const uint8_t* phase;
    const double* mat;     // per-phase constants, nparam each
    const float* mat32;    // the same table in float (float kernels read no doubles)
    const float* mat32lo;  // and the remainders, mat - mat32, for double-word constants
    int nparam;
    // grid constants in both precisions, so that no kernel converts them per element
    // (conversions and double arithmetic share the FP64 pipe, 1/64 of the FP32 rate)
    double half_n64, scale64, two_nsq64;  // N/2 (gradient stencil), 2/V (solve), 2 N^2 (Frank force)
    float half_n32, scale32, two_nsq32;
    // LCE directors (3 x V each, null for the other laws): ping-pong fields and the
    // reference directors n0, in both precisions
    double* N64[2];
    const double* n0_64;
    float* N32[2];
    const float* n0_32;
    // the previous time step of the LCE dissipation terms (F: d*d*V, n: 3*V): the state a
    // solve starts from, saved by launch_save_prev
    double *Fp64, *np64;
    float *Fp32, *np32;
    // double precision state
    double* F64[2];
    double* L64;
    double* U64[2];
    const double2* tw64;   // exp(-2 pi i m / N), m < N
    const double* ksq64;   // (N sin(2 pi m / N))^2, exact 0 at m = 0, N/2
    // single precision state
    float* F32[2];
    float* L32;
    float* U32[2];
    const float2* tw32;
    const float* ksq32;
    // double polish of RVE_MIXED: float increment R = F_{k+1} - G_k (d*d*V) and
    // its float spectrum (d*V); both alias float state buffers idle in that phase
    float* R32;
    float* S32;
    float* D32;  // float u~ increment of the last increment projection (d*V)
    // float phase of RVE_MIXED, 3D neo-Hookean with exact local steps on N = 128, 256, 512:
    // the z pass keeps the solved spectrum u^ (d * V/2 complex, in the idle double u~
    // buffer) and the squared norm of its change, so that the local pass takes r_d from
    // it (Parseval) instead of a second u~ stencil; zpart: one double per z-pass tile
    // (nz of them).  Null otherwise.
    float* Sprev;
    double* zpart;
    int nz;
    float *LH32, *LL32;  // Lambda as double-word (hi, lo) during the polish (idle float buffers)
    FftPlan plan;
};

// Per-iteration kernels run as persistent loops over a tile table: entry t is
// (RVE index into the descriptor array, block index within that RVE's grid for
// the pass).  An RVE's blocks, partial sums and reductions depend on its own size
// only, so its results are the same alone or in any batch.
enum TileClass : int { kTilesLocal = 0, kTilesX = 1, kTilesAx64 = 2, kTilesAx32 = 3, kTileClasses = 4 };

struct Exec {
    cudaStream_t stream;
    const Launch* rep;            // host copy of one member (dim, model, precision set)
    const Launch* rds;            // device array of member descriptors
    const int2* tiles[kTileClasses];
    int ntiles[kTileClasses];
    size_t smem_x[2];             // dynamic shared memory of the x passes [fp64], max over members
    size_t smem_a[2];             // and of the y/z passes
    int uniform_n;                // N shared by every member (0 if sizes differ)
    int uniform_geom;             // 1: every member has the first one's FFT geometry (lpb, tk)
    int exact_local;              // 1: no member takes approximate local steps (local_ratio,
                                  // local_fraction both 0): the float neo-Hookean law in 3D
                                  // then runs its closed-form local step
    // the members in tile-table order: host copies of their descriptors, whether each takes
    // exact local steps, and the index of each one's first tile in tiles[kTilesLocal].  In
    // launches of one grid size N = 128, 256 or 512 the fused local pass of the float
    // neo-Hookean law in 3D runs per member (k_local_cf for exact local steps), so that a
    // member's kernel does not depend on the others
    int nmem;
    const Launch* const* mem;
    const unsigned char* mem_exact;
    const int* mem_tile0;
};

// FFT geometry of one grid shape: x-pass lines per block and half-length radices,
// y/z tile widths and full-length radices (default rule or picked by the autotuner)
struct Geometry {
    int lpb, tk64, tk32;
    int np_half, np_full;
    int rad_half[kMaxPasses];
    int rad_full[kMaxPasses];
};
int factor_radices(int L, int* rad);
Geometry default_geometry(int dim, int n);
void register_geometry(int dim, int n, const Geometry& g);
bool lookup_geometry(int dim, int n, Geometry* g);
void apply_geometry(Launch& L, const Geometry& g);
// per-RVE launch geometry (local_blocks, lpb, xblocks, tk, radices) from dim and n
// (the registered tuned geometry of the shape if any, else the default rule)
void set_geometry(Launch& L);
// tiles of one RVE for each class
int tiles_local(const Launch& L);
int tiles_x(const Launch& L);
int tiles_ax(const Launch& L, bool fp64);
// dynamic shared memory of the x passes and of the y/z passes for one RVE
size_t smem_x_bytes(const Launch& L, bool fp64);
size_t smem_a_bytes(const Launch& L, bool fp64);
// grid size of a persistent launch: min(tiles, resident blocks on the device)
int persistent_grid(const void* kernel, int threads, size_t smem, int ntiles);

// rve_local.cu
cudaError_t launch_init(const Launch& L, bool fp64, bool lambda_zero);
// polish_mode (double only): 0 plain; 1 also write R; 2 also write R and take
// r_d from the float u~ increment D32 (see local_tile).
cudaError_t launch_local(const Exec& E, bool fp64, bool first, bool only_if_rho_changed, int polish_mode = 0);
// whether a member's fused local pass takes the lean per-RVE kernel (float phase, or the
// double-word polish with polish = true); the engine puts the other members' local tiles first
bool lean_local(const Launch& L, bool exact, bool polish);
cudaError_t launch_stress(const Launch& L, bool fp64);
// LCE: save the current state (F_k, n_k) as the previous time step, in every precision held
cudaError_t launch_save_prev(const Launch& L, bool from_fp64, cudaStream_t st);
// mixed macroscopic control: free components of <F> from the mean of F - Lambda/rho
// (dws: the state is in the double-word form of the polish)
cudaError_t launch_macro(const Launch& L, bool fp64, cudaStream_t st, bool dws = false);
// double <-> double-word state at the ends of the polish of the elastic laws
cudaError_t launch_polish_state(const Launch& L, bool enter, cudaStream_t st);
// RVE_MIXED, elastic laws without free <F> components: enter the double-word polish
// straight from the float state (F_{k+1}, Lambda_k, u~_k at ctrl->k = k), see rve_local.cu
cudaError_t launch_switch_direct(const Launch& L, cudaStream_t st);
cudaError_t launch_convert(const Launch& L, bool to_fp64);
// rve_fft.cu
cudaError_t launch_fft(const Exec& E, bool fp64, int stage = -1);
// whether FFT stage `stage` issues no kernel (folded into a fused neighbour)
bool fft_stage_empty(const Exec& E, bool fp64, int stage);
// Projection of the float increment R into the double u~: u~_{k+1} = u~_k + P(R).
cudaError_t launch_fft_incr(const Exec& E, int stage = -1);
inline int fft_stages(int dim) { return dim == 3 ? 5 : 3; }
cudaError_t prepare_fft_kernels(int n);

// ------------------------------------------------------------------ Bloch-wave ADMM (rve_bloch.cu)
struct BlochWork;  // device workspace, kept by the handle between calls
struct BlochArgs {
    int dim, n;
    long long V;
    int model;            // kNeoHooke or kLinear: L = W_FF(F) of the phase table
    const void* F;        // resident deformation gradient (d*d*V, double or float)
    bool F_fp64;
    const uint8_t* phase;
    const double* mat;
    int nparam;
    int k[3];             // Bloch wave numbers, omega_j = 2 pi / k_j
    double rho, tol, mu_ref;
    bool adaptive;        // Section 2.1's residual balancing of rho
    bool float_bulk;      // a float phase first (RVE_MIXED, RVE_FP32)
    bool promote;         // then FP64 to the tolerance (RVE_MIXED)
    double rho_kappa, rho_tau, rho_min;
    int max_iter, check_every;
    const double* p0;     // host, 2 d V doubles (re, im), component-major
    double* p_out;        // host or null
    double* hist_out;     // host (r_p, r_d, sigma, rho per iteration) or null
    cudaStream_t stream;
};
struct BlochResult {
    int iterations, float_iterations, converged, fail;
    double beta, rayleigh, r_p, r_d, time_ms, rho;
    long long launches;
};
int bloch_run(BlochWork** w, const BlochArgs& in, BlochResult* res);
void bloch_free(BlochWork* w);

}  // namespace admm
