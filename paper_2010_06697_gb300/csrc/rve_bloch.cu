// Bloch-wave ADMM for the modulus of stability (Section 2.4, Steps 1'-4').
//
// beta_k = min over unit Bloch waves v = p(x) exp(i omega.x), omega_j = 2 pi / k_j,
// of <grad v, L grad v>, with L(x) = W_FF(F(x)) of the resident state and the
// central differences of the periodic problem.  On the grid (h = 1/N) the central
// difference of v is exp(i omega.x) D p,
//   (D p)_ij(x) = (p_i(x + h e_j) e^{i th_j} - p_i(x - h e_j) e^{-i th_j}) / (2h),  th_j = omega_j h,
// with Fourier symbol i s_j(m), s_j(m) = N sin(2 pi (m_j + 1/k_j) / N).  One iteration:
//   1'. G = (L + rho I)^{-1} (g + rho D p)                      per voxel (Cholesky factor
//       of L + rho I computed once per call, double)
//   2'. p = argmin over ||p|| = 1 of rho/2 ||D p - Q||^2, Q = G - g/rho: in Fourier
//       p^ = rho b^ / (rho kappa - sigma), b = D^* Q, kappa = |s|^2, sigma below
//       rho min kappa the root of ||p|| = 1 (Newton passes on the spectrum with a
//       bisection safeguard)
//   3'. g += rho (D p - G)
//   4'. r_p = ||D p - G||, r_d = rho / mu_ref ||D (p - p_old)||.
// Fields are complex (float2 or double2), component-major (c * V + v), x fastest.
// Precision: FP64 throughout, or (handle precision RVE_MIXED / RVE_FP32) a float bulk --
// fields, factor, FFTs and the fused step in float; the spectrum weights, the Step 2'
// root, residuals and their sums in double -- promoted to FP64 (p and g converted, the
// factor and Step 1' redone in double) once the float residuals reach the float
// rounding level, as in the solver's RVE_MIXED.  The complex FFTs are this file's own:
// one block per tile of lines along an axis, the line in shared memory, Stockham
// radix-4/2/3 passes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "rve.h"
#include "rve_internal.cuh"

namespace admm {

struct BlochWork {
    size_t bytes = 0;
    unsigned char* base = nullptr;
    void* hctrl = nullptr;  // pinned mirror of the control block
    int max_hist = 0;
};

namespace {

constexpr int kBT = 256;            // threads per block
constexpr int kBlochBlocks = 1216;  // 152 SMs x 8: grid of the element-wise kernels
// Step 2' Newton passes per iteration (early exit): the first iterations start far
// from the root, later ones from the previous sigma
constexpr int kRootPasses0 = 32, kRootPasses1 = 16, kRootPasses = 8;
constexpr double kPi = 3.141592653589793238462643383279502884;

struct BCtrl {
    double sigma, lo, hi, pole;
    double rp, rd;
    double rho;        // penalty of the current iteration
    int rho_changed;   // set by the rule after an iteration, cleared by the next k_bdiv
    long long k;       // iterations done
    int stop;          // 1 converged, 3 non-finite residual
    int root_done;     // Step 2' root of the current iteration found
    int fail;          // bits: 1 L + rho I not positive definite, 2 no weight at the lowest
                       //       kappa (Step 2' hard case), 4 root passes exhausted
    unsigned counter;  // last-block detection of the reductions
};

struct FftPlanB {
    int n, npass, tl;
    int radix[12];
};

template <typename T>
struct Cx;
template <>
struct Cx<double> {
    using type = double2;
    __host__ __device__ static double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Cx<float> {
    using type = float2;
    __host__ __device__ static float2 make(float x, float y) { return make_float2(x, y); }
};

// Kernel arguments for fields of precision T (the spectrum weights, partial sums,
// history and symbol table are double in both).
template <typename T>
struct BArgs {
    using C = typename Cx<T>::type;
    int n, V;
    double tol, inv_mu_ref;
    int adaptive;          // Section 2.1's residual balancing of rho
    double kappa, tau, rho_floor;
    T c[3], s[3];          // cos, sin of th_j, times 1/(2h)
    const double* sym;     // s_j(m) at sym[j * n + m]
    const double* K;       // kappa(m) per frequency (k_bkappa, once per call)
    C *P0, *P1, *B, *G, *g, *Q;
    T *Lf, *Linv;
    double *W, *part, *hist;
    BCtrl* ctrl;
    int max_hist;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C, typename S>
__device__ __forceinline__ C cscale(C a, S s) { return C{a.x * s, a.y * s}; }

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double bwarp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Sum (or min) of NV values per thread over the block; the result is valid in thread 0.
template <int NV, bool MIN = false>
__device__ __forceinline__ void block_reduce(double* v) {
    __shared__ double s[kBT / 32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double r = MIN ? bwarp_min(v[q]) : bwarp_sum(v[q]);
        if (lane == 0) s[w][q] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double a = s[0][q];
            for (int i = 1; i < kBT / 32; ++i) a = MIN ? fmin(a, s[i][q]) : a + s[i][q];
            v[q] = a;
        }
    __syncthreads();
}

// Block partials to part[block * 4 + q]; returns true in thread 0 of the last block,
// whose v[] then holds the totals.  The last block reads the partials with all its
// threads (a fixed assignment, so the order of the sums is fixed) and reduces them.
template <int NV, bool MIN = false>
__device__ __forceinline__ bool grid_reduce(double* v, double* part, BCtrl* ctrl) {
    __shared__ int s_last;
    block_reduce<NV, MIN>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) part[blockIdx.x * 4 + q] = v[q];
        __threadfence();
        s_last = atomicAdd(&ctrl->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = MIN ? 1e300 : 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kBT)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = MIN ? fmin(v[q], __ldcg(part + b * 4 + q)) : v[q] + __ldcg(part + b * 4 + q);
    block_reduce<NV, MIN>(v);
    if (threadIdx.x != 0) return false;
    ctrl->counter = 0u;
    return true;
}

// Periodic neighbours of voxel v along each direction (x fastest).
template <int D>
__device__ __forceinline__ void bneighbours(int v, int n, int* up, int* dn) {
    const int x = v % n, r = v / n;
    up[0] = v + (x + 1 == n ? 1 - n : 1);
    dn[0] = v + (x == 0 ? n - 1 : -1);
    const int y = D == 3 ? r % n : r;
    up[1] = v + (y + 1 == n ? (1 - n) * n : n);
    dn[1] = v + (y == 0 ? (n - 1) * n : -n);
    if (D == 3) {
        const int z = r / n, s2 = n * n;
        up[2] = v + (z + 1 == n ? (1 - n) * s2 : s2);
        dn[2] = v + (z == 0 ? (n - 1) * s2 : -s2);
    }
}

// (D X)_ij at v for one (i, j).
template <typename T>
__device__ __forceinline__ typename Cx<T>::type bloch_grad1(const typename Cx<T>::type* __restrict__ X,
                                                            const BArgs<T>& a, int i, int j, int up, int dn) {
    const auto u = X[(size_t)i * a.V + up], w = X[(size_t)i * a.V + dn];
    const T c = a.c[j], s = a.s[j];
    return Cx<T>::make((u.x * c - u.y * s) - (w.x * c + w.y * s), (u.x * s + u.y * c) - (w.y * c - w.x * s));
}

// (D X)_ij at v from the neighbours of X (d complex components).
template <int D, typename T>
__device__ __forceinline__ void bloch_grad(const typename Cx<T>::type* __restrict__ X, const BArgs<T>& a,
                                           const int* up, const int* dn, typename Cx<T>::type* out) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) out[i * D + j] = bloch_grad1<T>(X, a, i, j, up[j], dn[j]);
}

// Packed lower-triangle index.
__host__ __device__ constexpr int tri(int p, int q) { return p * (p + 1) / 2 + q; }

// (L + rho I) x = b by the stored factor (real L, complex x and b).
template <int NN, typename T, typename C>
__device__ __forceinline__ void fsolve(const BArgs<T>& a, int v, const C* b, C* x) {
    C y[NN];
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        C s = b[p];
#pragma unroll
        for (int r = 0; r < p; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x -= l * y[r].x;
            s.y -= l * y[r].y;
        }
        y[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
#pragma unroll
    for (int p = NN - 1; p >= 0; --p) {
        C s = y[p];
#pragma unroll
        for (int r = p + 1; r < NN; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x -= l * x[r].x;
            s.y -= l * x[r].y;
        }
        x[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
}

// (L + rho I) x = b in place (forward substitution into b, then backward).
template <int NN, typename T, typename C>
__device__ __forceinline__ void fsolve_inplace(const BArgs<T>& a, int v, C* b) {
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        C s = b[p];
#pragma unroll
        for (int r = 0; r < p; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x -= l * b[r].x;
            s.y -= l * b[r].y;
        }
        b[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
#pragma unroll
    for (int p = NN - 1; p >= 0; --p) {
        C s = b[p];
#pragma unroll
        for (int r = p + 1; r < NN; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x -= l * b[r].x;
            s.y -= l * b[r].y;
        }
        b[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
}

// y = (L + rho I) x = F (F^T x) with the stored factor F.
template <int NN, typename T, typename C>
__device__ __forceinline__ void fapply(const BArgs<T>& a, int v, const C* x, C* y) {
    C t[NN];
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        C s{T(0), T(0)};
#pragma unroll
        for (int r = p; r < NN; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x += l * x[r].x;
            s.y += l * x[r].y;
        }
        t[p] = s;
    }
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        C s{T(0), T(0)};
#pragma unroll
        for (int r = 0; r <= p; ++r) {
            const T l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x += l * t[r].x;
            s.y += l * t[r].y;
        }
        y[p] = s;
    }
}

// kappa(m) = sum_j s_j(m_j)^2 with explicit roundings (no contraction), so that every
// kernel forms the same value.
template <int D, typename T>
__device__ __forceinline__ double kappa_calc(const BArgs<T>& a, int v) {
    const int n = a.n;
    const int mx = v % n, r = v / n;
    const int my = D == 3 ? r % n : r;
    const double sx = __ldg(a.sym + mx), sy = __ldg(a.sym + n + my);
    double k = __dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy));
    if (D == 3) {
        const double sz = __ldg(a.sym + 2 * n + r / n);
        k = __dadd_rn(k, __dmul_rn(sz, sz));
    }
    return k;
}

template <int D, typename T>
__device__ __forceinline__ double kappa_of(const BArgs<T>& a, int v) {
    return __ldg(a.K + v);
}

// ------------------------------------------------------------------ kernels
// Every kernel takes rho from the control block: the adaptive rule changes it between
// iterations.

// The table of kappa(m) the spectrum passes read.
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_bkappa(BArgs<T> a, double* K) {
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) K[v] = kappa_calc<D, T>(a, v);
}

// L + rho I = W_FF(F) + rho I per voxel (compressible neo-Hookean, Section 4.1, or
// isotropic linear elasticity), Cholesky-factored in double.
// mode 0: factor with ctrl->rho; mode 1: the same, only when rho changed (redo after the
// rule); mode 2: no factor stored, only the positive-definiteness test of L + shift I
// (fail bit 1), for the floor's bisection.
template <int D, int MODEL, typename TF, typename T>
__global__ void __launch_bounds__(kBT) k_bfactor(BArgs<T> a, const TF* __restrict__ F, const uint8_t* __restrict__ phase,
                                                 const double* __restrict__ mat, int nparam, int mode, double shift) {
    constexpr int NN = D * D;
    if (mode == 1 && !a.ctrl->rho_changed) return;
    const double rho = mode == 2 ? shift : a.ctrl->rho;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        const int ph = phase[v];
        const double mu = __ldg(mat + ph * nparam), lam = __ldg(mat + ph * nparam + 1);
        double H[NN * (NN + 1) / 2];
        if (MODEL == kNeoHooke) {
            double Fv[NN], A[NN];
#pragma unroll
            for (int p = 0; p < NN; ++p) Fv[p] = (double)F[(size_t)p * a.V + v];
            double J;
            if (D == 2) {
                J = Fv[0] * Fv[3] - Fv[1] * Fv[2];
                A[0] = Fv[3];
                A[1] = -Fv[2];
                A[2] = -Fv[1];
                A[3] = Fv[0];
            } else {
                A[0] = Fv[4] * Fv[8] - Fv[5] * Fv[7];
                A[1] = Fv[5] * Fv[6] - Fv[3] * Fv[8];
                A[2] = Fv[3] * Fv[7] - Fv[4] * Fv[6];
                A[3] = Fv[2] * Fv[7] - Fv[1] * Fv[8];
                A[4] = Fv[0] * Fv[8] - Fv[2] * Fv[6];
                A[5] = Fv[1] * Fv[6] - Fv[0] * Fv[7];
                A[6] = Fv[1] * Fv[5] - Fv[2] * Fv[4];
                A[7] = Fv[2] * Fv[3] - Fv[0] * Fv[5];
                A[8] = Fv[0] * Fv[4] - Fv[1] * Fv[3];
                J = Fv[0] * A[0] + Fv[1] * A[1] + Fv[2] * A[2];
            }
            const double iJ = 1.0 / J;
#pragma unroll
            for (int p = 0; p < NN; ++p) A[p] *= iJ;  // F^{-T}
            const double c = lam * J * (J - 1.0) - mu, b = lam * (2.0 * J - 1.0) * J;
            // W_FF[ij,kl] = mu d_ik d_jl + b A_ij A_kl - c A_il A_kj
#pragma unroll
            for (int p = 0; p < NN; ++p) {
                const int i = p / D, j = p % D;
#pragma unroll
                for (int q = 0; q <= p; ++q) {
                    const int k = q / D, l = q % D;
                    double h = b * A[p] * A[q] - c * A[i * D + l] * A[k * D + j];
                    if (p == q) h += mu + rho;
                    H[tri(p, q)] = h;
                }
            }
        } else {
            // mu (d_ik d_jl + d_il d_jk) + lam d_ij d_kl
#pragma unroll
            for (int p = 0; p < NN; ++p) {
                const int i = p / D, j = p % D;
#pragma unroll
                for (int q = 0; q <= p; ++q) {
                    const int k = q / D, l = q % D;
                    double h = mu * (double(i == k && j == l) + double(i == l && j == k)) + lam * double(i == j && k == l);
                    if (p == q) h += rho;
                    H[tri(p, q)] = h;
                }
            }
        }
        bool ok = true;
#pragma unroll
        for (int p = 0; p < NN; ++p) {
#pragma unroll
            for (int q = 0; q <= p; ++q) {
                double s = H[tri(p, q)];
#pragma unroll
                for (int r = 0; r < q; ++r) s -= H[tri(p, r)] * H[tri(q, r)];
                if (p == q) {
                    ok = ok && s > 0.0;
                    const double d = sqrt(fmax(s, 0.0));
                    H[tri(p, p)] = d;
                    if (mode != 2) a.Linv[(size_t)p * a.V + v] = (T)(ok ? 1.0 / d : 0.0);
                } else {
                    H[tri(p, q)] = s / H[tri(q, q)];
                }
            }
        }
        if (!ok) {
            atomicOr(&a.ctrl->fail, 1);
#pragma unroll
            for (int p = 0; p < NN * (NN + 1) / 2; ++p) H[p] = 0.0;
        }
        if (mode == 2) continue;
#pragma unroll
        for (int p = 0; p < NN * (NN + 1) / 2; ++p) a.Lf[(size_t)p * a.V + v] = (T)H[p];
    }
}

// Start: g_0 = L D p_0, then Step 1' of the first iteration (G, Q).
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_binit(BArgs<T> a) {
    constexpr int NN = D * D;
    using C = typename Cx<T>::type;
    const T rho = (T)a.ctrl->rho, inv_rho = (T)(1.0 / a.ctrl->rho);
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        C Dp[NN], y[NN], rhs[NN], G[NN];
        bloch_grad<D, T>(a.P0, a, up, dn, Dp);
        fapply<NN>(a, v, Dp, y);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            const C g0 = csub(y[p], cscale(Dp[p], rho));
            y[p] = g0;
            rhs[p] = cadd(g0, cscale(Dp[p], rho));
        }
        fsolve<NN>(a, v, rhs, G);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.g[(size_t)p * a.V + v] = y[p];
            a.G[(size_t)p * a.V + v] = G[p];
            a.Q[(size_t)p * a.V + v] = Cx<T>::make(G[p].x - y[p].x * inv_rho, G[p].y - y[p].y * inv_rho);
        }
    }
}

// b = D^* Q: (D^* Q)_i = sum_j (Q_ij(x - h e_j) e^{-i th_j} - Q_ij(x + h e_j) e^{i th_j}) / (2h).
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_bdiv(BArgs<T> a) {
    if (a.ctrl->stop) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->rho_changed = 0;  // the redo (if any) has run
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            T re = T(0), im = T(0);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const auto w = a.Q[(size_t)(i * D + j) * a.V + dn[j]], u = a.Q[(size_t)(i * D + j) * a.V + up[j]];
                const T c = a.c[j], s = a.s[j];
                re += (w.x * c + w.y * s) - (u.x * c - u.y * s);
                im += (w.y * c - w.x * s) - (u.x * s + u.y * c);
            }
            a.B[(size_t)i * a.V + v] = Cx<T>::make(re, im);
        }
    }
}

// In-place complex FFT of the d components of B along one axis.  A block takes a tile
// of tl lines (consecutive rows for the x axis, consecutive x (or x-y plane
// positions) for the others, so that loads coalesce), holds it in shared memory and
// runs Stockham passes of radix 4, 2 and 3 (tw[t] = exp(-2 pi i t / n)).
template <int D, int AXIS, bool INV, typename T>
__global__ void __launch_bounds__(kBT) k_bfft(BArgs<T> a, const typename Cx<T>::type* __restrict__ tw, FftPlanB pl) {
    using C = typename Cx<T>::type;
    if (a.ctrl->stop) return;
    extern __shared__ __align__(16) unsigned char bsm_raw[];
    C* bsm = reinterpret_cast<C*>(bsm_raw);
    const int n = pl.n, tl = pl.tl;
    const int nl = a.V / n;
    const int ntile = (nl + tl - 1) / tl;
    C* s0 = bsm;
    C* s1 = bsm + tl * n;
    auto addr = [&](int line, int i) -> size_t {
        if (AXIS == 0) return (size_t)line * n + i;
        if (AXIS == 1) {
            if (D == 2) return (size_t)i * n + line;
            const int z = line / n, x = line - z * n;
            return ((size_t)z * n + i) * n + x;
        }
        return (size_t)i * n * n + line;
    };
    for (int tile = blockIdx.x; tile < ntile * D; tile += gridDim.x) {
        const int comp = tile / ntile, t0 = (tile - comp * ntile) * tl;
        C* base = a.B + (size_t)comp * a.V;
        for (int t = threadIdx.x; t < tl * n; t += kBT) {
            int l, i;
            if (AXIS == 0) {
                l = t / n;
                i = t - l * n;
            } else {
                i = t / tl;
                l = t - i * tl;
            }
            if (t0 + l < nl) s0[l * n + i] = base[addr(t0 + l, i)];
        }
        __syncthreads();
        C* in = s0;
        C* out = s1;
        int ns = 1;
        for (int ps = 0; ps < pl.npass; ++ps) {
            const int R = pl.radix[ps], m = n / R, tws = n / (ns * R);
            for (int t = threadIdx.x; t < tl * m; t += kBT) {
                const int l = t / m, j = t - l * m, kk = j % ns;
                const C* li = in + l * n;
                C* lo = out + l * n;
                const int o = (j - kk) * R + kk;
                C x0 = li[j], x1 = li[j + m];
                if (kk) {
                    C w = tw[kk * tws];
                    if (INV) w.y = -w.y;
                    x1 = cmul(x1, w);
                }
                if (R == 2) {
                    lo[o] = cadd(x0, x1);
                    lo[o + ns] = csub(x0, x1);
                } else if (R == 3) {
                    C x2 = li[j + 2 * m];
                    if (kk) {
                        C w = tw[2 * kk * tws];
                        if (INV) w.y = -w.y;
                        x2 = cmul(x2, w);
                    }
                    // y1,2 = x0 - (x1 + x2)/2 -+ i sqrt(3)/2 (x1 - x2) (forward; signs swap inverse)
                    const T h3 = INV ? T(-0.86602540378443864676) : T(0.86602540378443864676);
                    const C t1 = cadd(x1, x2), t2 = csub(x1, x2);
                    const C mid = Cx<T>::make(x0.x - T(0.5) * t1.x, x0.y - T(0.5) * t1.y);
                    lo[o] = cadd(x0, t1);
                    lo[o + ns] = Cx<T>::make(mid.x + h3 * t2.y, mid.y - h3 * t2.x);
                    lo[o + 2 * ns] = Cx<T>::make(mid.x - h3 * t2.y, mid.y + h3 * t2.x);
                } else {
                    C x2 = li[j + 2 * m], x3 = li[j + 3 * m];
                    if (kk) {
                        C w2 = tw[2 * kk * tws], w3 = tw[3 * kk * tws];
                        if (INV) {
                            w2.y = -w2.y;
                            w3.y = -w3.y;
                        }
                        x2 = cmul(x2, w2);
                        x3 = cmul(x3, w3);
                    }
                    // y0 = a0+a1+a2+a3, y2 = a0-a1+a2-a3, y1,3 = (a0-a2) -+ i (a1-a3) (forward)
                    const C e = cadd(x0, x2), f = csub(x0, x2), g2 = cadd(x1, x3), h = csub(x1, x3);
                    lo[o] = cadd(e, g2);
                    lo[o + 2 * ns] = csub(e, g2);
                    if (!INV) {
                        lo[o + ns] = Cx<T>::make(f.x + h.y, f.y - h.x);
                        lo[o + 3 * ns] = Cx<T>::make(f.x - h.y, f.y + h.x);
                    } else {
                        lo[o + ns] = Cx<T>::make(f.x - h.y, f.y + h.x);
                        lo[o + 3 * ns] = Cx<T>::make(f.x + h.y, f.y - h.x);
                    }
                }
            }
            __syncthreads();
            C* sw = in;
            in = out;
            out = sw;
            ns *= R;
        }
        for (int t = threadIdx.x; t < tl * n; t += kBT) {
            int l, i;
            if (AXIS == 0) {
                l = t / n;
                i = t - l * n;
            } else {
                i = t / tl;
                l = t - i * tl;
            }
            if (t0 + l < nl) base[addr(t0 + l, i)] = in[l * n + i];
        }
        __syncthreads();
    }
}

// W(m) = sum_i |b^_i(m)|^2, with sum W, min kappa and W_min, the sum of W where kappa
// is minimal.  The last block brackets the root of ||p(sigma)|| = 1 below the pole
// rho min kappa: lo = pole - 2 rho sqrt(sum W) / V has ||p|| <= 1/2, and
// sigma_R = pole - rho sqrt(W_min) / V has ||p|| >= 1 (its W_min terms alone reach 1),
// so the root lies in [lo, sigma_R]; Newton starts from the previous sigma when it
// lies inside, else from sigma_R (where phi is concave and Newton is monotone).
__device__ __forceinline__ void kw_merge(double& k, double& w, double k2, double w2) {
    if (k2 < k) {
        k = k2;
        w = w2;
    } else if (k2 == k) {
        w += w2;
    }
}

// Block-wide (sum of ws, merge of (km, wm)); valid in thread 0.
__device__ __forceinline__ void block_merge3(double& ws, double& km, double& wm) {
    __shared__ double s3[kBT / 32][3];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ws += __shfl_down_sync(0xffffffffu, ws, o);
        const double k2 = __shfl_down_sync(0xffffffffu, km, o), w2 = __shfl_down_sync(0xffffffffu, wm, o);
        kw_merge(km, wm, k2, w2);
    }
    if (lane == 0) {
        s3[wi][0] = ws;
        s3[wi][1] = km;
        s3[wi][2] = wm;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < kBT / 32; ++i) {
            ws += s3[i][0];
            kw_merge(km, wm, s3[i][1], s3[i][2]);
        }
    __syncthreads();
}

template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_bweights(BArgs<T> a) {
    if (a.ctrl->stop) return;
    double ws = 0.0, km = 1e300, wm = 0.0;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        T wt = T(0);  // in the field precision: the spectrum of a float phase is float
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const auto b = a.B[(size_t)i * a.V + v];
            wt += b.x * b.x + b.y * b.y;
        }
        const double w = (double)wt;
        a.W[v] = w;
        ws += w;
        kw_merge(km, wm, kappa_of<D, T>(a, v), w);
    }
    __shared__ int s_last;
    block_merge3(ws, km, wm);
    if (threadIdx.x == 0) {
        a.part[blockIdx.x * 4 + 0] = ws;
        a.part[blockIdx.x * 4 + 1] = km;
        a.part[blockIdx.x * 4 + 2] = wm;
        __threadfence();
        s_last = atomicAdd(&a.ctrl->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    ws = 0.0;
    km = 1e300;
    wm = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kBT) {
        ws += __ldcg(a.part + b * 4);
        kw_merge(km, wm, __ldcg(a.part + b * 4 + 1), __ldcg(a.part + b * 4 + 2));
    }
    block_merge3(ws, km, wm);
    if (threadIdx.x != 0) return;
    BCtrl* c = a.ctrl;
    c->counter = 0u;
    const double rho = c->rho;
    const double pole = __dmul_rn(rho, km), Vd = (double)a.V;
    const double lo = pole - 2.0 * rho * sqrt(ws) / Vd;
    const double sr = fmin(pole - rho * sqrt(wm) / Vd, nextafter(pole, -1e300));
    c->pole = pole;
    c->root_done = 0;
    if (!(wm > 0.0) || !(lo < sr)) {  // no weight at the lowest kappa: the hard case
        c->root_done = 1;
        c->fail |= 2;
        c->stop = 3;
        return;
    }
    c->lo = lo;
    c->hi = sr;
    const double sp = c->sigma;
    c->sigma = (sp > lo && sp < sr) ? sp : sr;
}

// One Newton pass on phi(sigma) = V / sqrt(S) - 1, S = sum rho^2 W / (rho kappa - sigma)^2
// (phi decreasing; phi = 0 is ||p|| = 1), keeping the bracket [lo, hi] of the root and
// bisecting when Newton leaves it.
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_broot(BArgs<T> a, int last) {
    const BCtrl* cc = a.ctrl;
    if (cc->stop || cc->root_done) return;
    const double sig = cc->sigma, rho = cc->rho, r2 = rho * rho;
    double v2[2] = {0.0, 0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        const double inv = 1.0 / __dsub_rn(__dmul_rn(rho, kappa_of<D, T>(a, v)), sig);
        const double q = r2 * a.W[v] * inv * inv;
        v2[0] += q;
        v2[1] += 2.0 * q * inv;
    }
    if (!grid_reduce<2>(v2, a.part, a.ctrl)) return;
    BCtrl* c = a.ctrl;
    const double S = v2[0], dS = v2[1], Vd = (double)a.V;
    const double phi = Vd / sqrt(S) - 1.0;
    if (phi == 0.0) {
        c->root_done = 1;
        return;
    }
    double lo = c->lo, hi = c->hi;
    if (phi > 0.0) lo = sig;
    else hi = sig;
    const double dphi = -0.5 * Vd * dS / (S * sqrt(S));
    double nxt = sig - phi / dphi;
    c->lo = lo;
    c->hi = hi;
    const double tolr = 4.0 * 2.220446049250313e-16 * fmax(fabs(sig), fabs(c->pole));
    if (fabs(nxt - sig) <= tolr) {  // the Newton step is at the rounding level: converged
        c->root_done = 1;
        if (nxt < c->pole) c->sigma = nxt;
        return;
    }
    if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);  // safeguard: bisect the bracket
    if (hi - lo <= tolr) {  // the bracket always holds the root
        c->root_done = 1;
    } else if (last) {
        c->fail |= 4;
        c->stop = 3;
    }
    c->sigma = nxt;
}

// p^ = rho b^ / (rho kappa - sigma), with the 1/V of the inverse transform.
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_bphat(BArgs<T> a) {
    if (a.ctrl->stop) return;
    const double sig = a.ctrl->sigma, rho = a.ctrl->rho, Vd = (double)a.V;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        const double den = __dsub_rn(__dmul_rn(rho, kappa_of<D, T>(a, v)), sig);
        const T f = (T)(rho / (den * Vd));
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const auto b = a.B[(size_t)i * a.V + v];
            a.B[(size_t)i * a.V + v] = Cx<T>::make(b.x * f, b.y * f);
        }
    }
}

// Steps 3' and 4' of iteration i (p_i in B, p_{i-1} in Pold, G_i, g_{i-1}) fused with
// Step 1' of iteration i + 1 (G_{i+1}, Q); p_i is copied to Pnew.  The last block
// finishes the residuals, records them and sets the stop flag.
template <int D, typename T>
__global__ void __launch_bounds__(kBT, (sizeof(T) == 4 || D == 2) ? 2 : 1)
k_blocal(BArgs<T> a, const typename Cx<T>::type* __restrict__ Pold, typename Cx<T>::type* __restrict__ Pnew) {
    constexpr int NN = D * D;
    using C = typename Cx<T>::type;
    if (a.ctrl->stop) return;
    const double rho = a.ctrl->rho;
    const T rho_t = (T)rho, inv_rho = (T)(1.0 / rho);
    double v2[2] = {0.0, 0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        C x[NN], gn[NN];
        T sp = T(0), sd = T(0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int p = i * D + j;
                const C Dn = bloch_grad1<T>(a.B, a, i, j, up[j], dn[j]);
                const C Do = bloch_grad1<T>(Pold, a, i, j, up[j], dn[j]);
                const C e = csub(Dn, a.G[(size_t)p * a.V + v]), dd = csub(Dn, Do);
                sp += e.x * e.x + e.y * e.y;
                sd += dd.x * dd.x + dd.y * dd.y;
                gn[p] = cadd(a.g[(size_t)p * a.V + v], cscale(e, rho_t));  // Step 3'
                x[p] = cadd(gn[p], cscale(Dn, rho_t));
            }
        v2[0] += (double)sp;  // per voxel in T, over voxels in double
        v2[1] += (double)sd;
        fsolve_inplace<NN>(a, v, x);  // Step 1' of the next iteration
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.g[(size_t)p * a.V + v] = gn[p];
            a.G[(size_t)p * a.V + v] = x[p];
            a.Q[(size_t)p * a.V + v] = Cx<T>::make(x[p].x - gn[p].x * inv_rho, x[p].y - gn[p].y * inv_rho);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) Pnew[(size_t)i * a.V + v] = a.B[(size_t)i * a.V + v];
    }
    if (!grid_reduce<2>(v2, a.part, a.ctrl)) return;
    BCtrl* c = a.ctrl;
    const double rp = sqrt(v2[0] / (double)a.V), rd = rho * a.inv_mu_ref * sqrt(v2[1] / (double)a.V);
    if (c->k < a.max_hist) {
        a.hist[4 * c->k] = rp;
        a.hist[4 * c->k + 1] = rd;
        a.hist[4 * c->k + 2] = c->sigma;
        a.hist[4 * c->k + 3] = rho;
    }
    c->k += 1;
    c->rp = rp;
    c->rd = rd;
    if (!(rp == rp) || !(rd == rd)) c->stop = 3;
    else if (rp <= a.tol && rd <= a.tol) c->stop = 1;
    else if (a.adaptive) {  // Section 2.1's rule; Step 1' of the next iteration is redone
        double nr = rho;
        if (rd > 0.0 && rp / rd > a.tau) nr = a.kappa * rho;
        else if (rp > 0.0 && rd / rp > a.tau) nr = fmax(rho / a.kappa, a.rho_floor);
        if (nr != rho) {
            c->rho = nr;
            c->rho_changed = 1;
        }
    }
}

// Step 1' again after the rule changed rho (the fused step used the old one):
// G = (L + rho I)^{-1} (g + rho D p), Q = G - g / rho with p in P and the new factor.
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_bredo(BArgs<T> a, const typename Cx<T>::type* __restrict__ P) {
    constexpr int NN = D * D;
    using C = typename Cx<T>::type;
    if (a.ctrl->stop || !a.ctrl->rho_changed) return;
    const T rho = (T)a.ctrl->rho, inv_rho = (T)(1.0 / a.ctrl->rho);
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        C x[NN], gv[NN];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int p = i * D + j;
                gv[p] = a.g[(size_t)p * a.V + v];
                x[p] = cadd(gv[p], cscale(bloch_grad1<T>(P, a, i, j, up[j], dn[j]), rho));
            }
        fsolve_inplace<NN>(a, v, x);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.G[(size_t)p * a.V + v] = x[p];
            a.Q[(size_t)p * a.V + v] = Cx<T>::make(x[p].x - gv[p].x * inv_rho, x[p].y - gv[p].y * inv_rho);
        }
    }
}

// Promotion of the float bulk to FP64: p (d components) and g (d^2) converted; the
// double factor and Step 1' are then redone (k_bfactor mode 1, k_bredo).
template <int D>
__global__ void __launch_bounds__(kBT) k_bpromote(const float2* __restrict__ pf, const float2* __restrict__ gf,
                                                  double2* __restrict__ pd, double2* __restrict__ gd, int V) {
    for (int v = blockIdx.x * kBT + threadIdx.x; v < V; v += gridDim.x * kBT) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float2 q = pf[(size_t)i * V + v];
            pd[(size_t)i * V + v] = make_double2(q.x, q.y);
        }
#pragma unroll
        for (int p = 0; p < D * D; ++p) {
            const float2 q = gf[(size_t)p * V + v];
            gd[(size_t)p * V + v] = make_double2(q.x, q.y);
        }
    }
}

// <D p, L D p> = mean over voxels of |F^T Dp|^2 - rho |Dp|^2 (F the stored factor).
template <int D, typename T>
__global__ void __launch_bounds__(kBT) k_brayleigh(BArgs<T> a, const typename Cx<T>::type* __restrict__ P, double* out) {
    constexpr int NN = D * D;
    using C = typename Cx<T>::type;
    const double rho = a.ctrl->rho;
    double v1[1] = {0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        C Dp[NN], y[NN];
        bloch_grad<D, T>(P, a, up, dn, Dp);
        fapply<NN>(a, v, Dp, y);
#pragma unroll
        for (int p = 0; p < NN; ++p)
            v1[0] += ((double)Dp[p].x * y[p].x + (double)Dp[p].y * y[p].y) -
                     rho * ((double)Dp[p].x * Dp[p].x + (double)Dp[p].y * Dp[p].y);
    }
    if (!grid_reduce<1>(v1, a.part, a.ctrl)) return;
    *out = v1[0] / (double)a.V;
}

// ------------------------------------------------------------------ host side

FftPlanB make_plan(int n) {
    FftPlanB p{};
    p.n = n;
    int m = n;
    while (m % 4 == 0) {
        p.radix[p.npass++] = 4;
        m /= 4;
    }
    while (m % 2 == 0) {
        p.radix[p.npass++] = 2;
        m /= 2;
    }
    while (m % 3 == 0) {
        p.radix[p.npass++] = 3;
        m /= 3;
    }
    p.tl = std::max(1, std::min(64, 2048 / n));
    return p;
}

int grid_for(long long V) { return (int)std::min<long long>(kBlochBlocks, (V + kBT - 1) / kBT); }

template <int D, typename T>
cudaError_t set_fft_attrs(size_t smem) {
    static size_t done = 0;
    if (done >= smem) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const int b = (int)smem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 0, false, T>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 0, true, T>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 1, false, T>, at, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 1, true, T>, at, b);
    if (D == 3) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, D - 1, false, T>, at, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, D - 1, true, T>, at, b);
    }
    if (e == cudaSuccess) done = smem;
    return e;
}

template <int D, bool INV, typename T>
void fft_all(const BArgs<T>& a, const typename Cx<T>::type* tw, const FftPlanB& pl, size_t smem, int fg,
             cudaStream_t st) {
    k_bfft<D, 0, INV, T><<<fg, kBT, smem, st>>>(a, tw, pl);
    k_bfft<D, 1, INV, T><<<fg, kBT, smem, st>>>(a, tw, pl);
    if (D == 3) k_bfft<D, D - 1, INV, T><<<fg, kBT, smem, st>>>(a, tw, pl);
}

// The launches of one precision phase: factor, init, iteration, graphs.
template <int D, typename T>
struct Phase {
    using C = typename Cx<T>::type;
    BArgs<T> a{};
    const BlochArgs* in = nullptr;
    C* tw = nullptr;
    FftPlanB pl{};
    size_t smem = 0;
    int eg = 0, fg = 0;
    cudaStream_t st = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int per_chunk = 0;

    void factor(int mode, double shift) const {
        const BlochArgs& b = *in;
        if (b.model == kNeoHooke) {
            if (b.F_fp64)
                k_bfactor<D, kNeoHooke, double, T><<<eg, kBT, 0, st>>>(a, (const double*)b.F, b.phase, b.mat, b.nparam,
                                                                       mode, shift);
            else
                k_bfactor<D, kNeoHooke, float, T><<<eg, kBT, 0, st>>>(a, (const float*)b.F, b.phase, b.mat, b.nparam,
                                                                      mode, shift);
        } else {
            if (b.F_fp64)
                k_bfactor<D, kLinear, double, T><<<eg, kBT, 0, st>>>(a, (const double*)b.F, b.phase, b.mat, b.nparam,
                                                                     mode, shift);
            else
                k_bfactor<D, kLinear, float, T><<<eg, kBT, 0, st>>>(a, (const float*)b.F, b.phase, b.mat, b.nparam,
                                                                    mode, shift);
        }
    }
    C* pold(long long i) const { return ((i - 1) & 1) ? a.P1 : a.P0; }
    C* pnew(long long i) const { return (i & 1) ? a.P1 : a.P0; }
    // iteration i (1-based, counted over both phases) reads p_{i-1} and writes p_i
    int iteration(long long i) const {
        const int passes = i == 1 ? kRootPasses0 : (i == 2 ? kRootPasses1 : kRootPasses);
        k_bdiv<D, T><<<eg, kBT, 0, st>>>(a);
        fft_all<D, false, T>(a, tw, pl, smem, fg, st);
        k_bweights<D, T><<<eg, kBT, 0, st>>>(a);
        for (int r = 0; r < passes; ++r) k_broot<D, T><<<eg, kBT, 0, st>>>(a, r == passes - 1);
        k_bphat<D, T><<<eg, kBT, 0, st>>>(a);
        fft_all<D, true, T>(a, tw, pl, smem, fg, st);
        k_blocal<D, T><<<eg, kBT, 0, st>>>(a, pold(i), pnew(i));
        if (a.adaptive) {  // after a change of rho: new factor, Step 1' again
            factor(1, 0.0);
            k_bredo<D, T><<<eg, kBT, 0, st>>>(a, pnew(i));
        }
        return 4 + 2 * D + passes + (a.adaptive ? 2 : 0);
    }
    // m iterations from it (plain launches, or the graph of this phase for the
    // starting parity once past the first two iterations); returns launches or -1
    long long chunk(long long it, long long m, int full) {
        if (it >= 2 && m == full) {
            const int par = (int)(it & 1);
            if (!graph[par]) {
                cudaGraph_t g = nullptr;
                per_chunk = 0;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
                for (long long q = 0; q < m; ++q) per_chunk += iteration(it + q + 1);
                const cudaError_t ec = cudaStreamEndCapture(st, &g);
                const cudaError_t ei = ec == cudaSuccess ? cudaGraphInstantiate(&graph[par], g, 0) : ec;
                if (g) cudaGraphDestroy(g);
                if (ei != cudaSuccess) return -1;
            }
            if (cudaGraphLaunch(graph[par], st) != cudaSuccess) return -1;
            return per_chunk;
        }
        long long l = 0;
        for (long long q = 0; q < m; ++q) l += iteration(it + q + 1);
        return l;
    }
    void drop() {
        for (auto& g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
};

template <int D, typename T>
void bind(Phase<D, T>& ph, unsigned char* b, size_t oP0, size_t oP1, size_t oB, size_t oG, size_t og, size_t oQ,
          size_t oL, size_t oLi, size_t otw) {
    using C = typename Cx<T>::type;
    ph.a.P0 = (C*)(b + oP0);
    ph.a.P1 = (C*)(b + oP1);
    ph.a.B = (C*)(b + oB);
    ph.a.G = (C*)(b + oG);
    ph.a.g = (C*)(b + og);
    ph.a.Q = (C*)(b + oQ);
    ph.a.Lf = (T*)(b + oL);
    ph.a.Linv = (T*)(b + oLi);
    ph.tw = (C*)(b + otw);
}

template <int D>
int run(BlochWork* w, const BlochArgs& in, BlochResult* res) {
    constexpr int NN = D * D;
    constexpr int NP = NN * (NN + 1) / 2;
    const int n = in.n;
    const long long V = in.V;
    cudaStream_t st = in.stream;
    const bool bulk = in.float_bulk;  // float phase first
    // workspace layout: the double set, the float set when there is a float phase, shared
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 255) / 256 * 256;
        return o;
    };
    const size_t dP0 = take(16 * D * V), dP1 = take(16 * D * V), dB = take(16 * D * V);
    const size_t dG = take(16 * NN * V), dg = take(16 * NN * V), dQ = take(16 * NN * V);
    const size_t dL = take(8 * (size_t)NP * V), dLi = take(8 * NN * V), dtw = take(16 * n);
    size_t fP0 = 0, fP1 = 0, fB = 0, fG = 0, fg_ = 0, fQ = 0, fL = 0, fLi = 0, ftw = 0;
    if (bulk) {
        fP0 = take(8 * D * V), fP1 = take(8 * D * V), fB = take(8 * D * V);
        fG = take(8 * NN * V), fg_ = take(8 * NN * V), fQ = take(8 * NN * V);
        fL = take(4 * (size_t)NP * V), fLi = take(4 * NN * V), ftw = take(8 * n);
    }
    const size_t oW = take(8 * V), oK = take(8 * V), opart = take(8 * 4 * kBlochBlocks),
                 ohist = take(8 * 4 * (size_t)in.max_iter);
    const size_t osym = take(8 * 3 * n), octrl = take(sizeof(BCtrl)), orq = take(8);
    if (w->bytes < off) {
        if (w->base) cudaFree(w->base);
        w->base = nullptr;
        w->bytes = 0;
        if (cudaMalloc((void**)&w->base, off) != cudaSuccess) return RVE_E_OOM;
        w->bytes = off;
    }
    if (!w->hctrl && cudaMallocHost(&w->hctrl, sizeof(BCtrl) + 64) != cudaSuccess) return RVE_E_OOM;
    unsigned char* b = w->base;

    const FftPlanB pl = make_plan(n);
    const int eg = grid_for(V);
    const int fgrid = std::min((int)((V / n + pl.tl - 1) / pl.tl) * D, 152 * 3);
    Phase<D, double> pd;
    Phase<D, float> pf;
    auto common = [&](auto& ph) {
        auto& a = ph.a;
        a.n = n;
        a.V = (int)V;
        a.tol = in.tol;
        a.inv_mu_ref = 1.0 / in.mu_ref;
        a.adaptive = in.adaptive ? 1 : 0;
        a.kappa = in.rho_kappa;
        a.tau = in.rho_tau;
        a.rho_floor = 0.0;
        for (int j = 0; j < 3; ++j) {
            const double th = j < D ? 2.0 * kPi / ((double)in.k[j] * n) : 0.0;
            a.c[j] = 0.5 * n * cos(th);
            a.s[j] = 0.5 * n * sin(th);
        }
        a.W = (double*)(b + oW);
        a.part = (double*)(b + opart);
        a.hist = (double*)(b + ohist);
        a.sym = (const double*)(b + osym);
        a.K = (const double*)(b + oK);
        a.ctrl = (BCtrl*)(b + octrl);
        a.max_hist = in.max_iter;
        ph.in = &in;
        ph.pl = pl;
        ph.eg = eg;
        ph.fg = fgrid;
        ph.st = st;
    };
    common(pd);
    bind(pd, b, dP0, dP1, dB, dG, dg, dQ, dL, dLi, dtw);
    pd.smem = (size_t)2 * pl.tl * n * sizeof(double2);
    if (bulk) {
        common(pf);
        bind(pf, b, fP0, fP1, fB, fG, fg_, fQ, fL, fLi, ftw);
        pf.smem = (size_t)2 * pl.tl * n * sizeof(float2);
    }
    double* d_rq = (double*)(b + orq);
    BCtrl* dctrl = pd.a.ctrl;

    // host-side tables and the normalised start
    std::vector<double> sym(3 * (size_t)n, 0.0);
    for (int j = 0; j < D; ++j)
        for (int m = 0; m < n; ++m) sym[(size_t)j * n + m] = n * sin(2.0 * kPi * (m + 1.0 / in.k[j]) / n);
    std::vector<double2> twh(n);
    std::vector<float2> twf(n);
    for (int t = 0; t < n; ++t) {
        twh[t] = make_double2(cos(2.0 * kPi * t / n), -sin(2.0 * kPi * t / n));
        twf[t] = make_float2((float)twh[t].x, (float)twh[t].y);
    }
    double nrm = 0.0;
    for (size_t i = 0; i < 2 * (size_t)D * V; ++i) nrm += in.p0[i] * in.p0[i];
    nrm = sqrt(nrm / (double)V);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return RVE_E_INVALID_ARG;
    std::vector<double> p0((size_t)2 * D * V);
    for (size_t i = 0; i < p0.size(); ++i) p0[i] = in.p0[i] / nrm;
    BCtrl c0{};
    c0.sigma = NAN;
    c0.rho = in.rho;
#define CKB(x)                                     \
    do {                                           \
        if ((x) != cudaSuccess) return RVE_E_CUDA; \
    } while (0)
    CKB(cudaMemcpyAsync((void*)pd.a.sym, sym.data(), sym.size() * 8, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(pd.tw, twh.data(), twh.size() * 16, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(dctrl, &c0, sizeof(BCtrl), cudaMemcpyHostToDevice, st));
    k_bkappa<D, double><<<eg, kBT, 0, st>>>(pd.a, (double*)(b + oK));
    CKB((set_fft_attrs<D, double>(pd.smem)));
    if (bulk) {
        std::vector<float> p0f(p0.size());
        for (size_t i = 0; i < p0.size(); ++i) p0f[i] = (float)p0[i];
        CKB(cudaMemcpyAsync(pf.tw, twf.data(), twf.size() * 8, cudaMemcpyHostToDevice, st));
        CKB(cudaMemcpyAsync(pf.a.P0, p0f.data(), p0f.size() * 4, cudaMemcpyHostToDevice, st));
        CKB((set_fft_attrs<D, float>(pf.smem)));
    } else {
        CKB(cudaMemcpyAsync(pd.a.P0, p0.data(), p0.size() * 8, cudaMemcpyHostToDevice, st));
    }
    long long launches = 1;  // k_bkappa
    BCtrl* hc = (BCtrl*)w->hctrl;
    auto read_ctrl = [&]() -> bool {
        return cudaGetLastError() == cudaSuccess &&
               cudaMemcpyAsync(hc, dctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess;
    };
    // positive definiteness at the starting rho (the double factor decides)
    pd.factor(0, 0.0);
    launches += 1;
    if (!read_ctrl()) return RVE_E_CUDA;
    if (hc->fail & 1) return RVE_E_NUMERICAL;
    if (in.adaptive) {
        // floor of the rule: max(rho_min or mu_ref, 2 s*), s* the smallest shift with
        // L + s* I positive definite everywhere (bisection on [0, rho], to 2^-16 rho)
        auto pdtest = [&](double sft) -> int {
            if (cudaMemsetAsync(&dctrl->fail, 0, sizeof(int), st) != cudaSuccess) return -1;
            pd.factor(2, sft);
            launches += 1;
            if (!read_ctrl()) return -1;
            return (hc->fail & 1) ? 0 : 1;
        };
        double smin = 0.0;
        const int r0 = pdtest(0.0);
        if (r0 < 0) return RVE_E_CUDA;
        if (!r0) {
            double lo = 0.0, hi = in.rho;
            for (int it = 0; it < 16; ++it) {
                const double mid = 0.5 * (lo + hi);
                const int r = pdtest(mid);
                if (r < 0) return RVE_E_CUDA;
                if (r) hi = mid;
                else lo = mid;
            }
            smin = hi;
        }
        CKB(cudaMemsetAsync(&dctrl->fail, 0, sizeof(int), st));
        pd.a.rho_floor = pf.a.rho_floor = std::max(in.rho_min > 0.0 ? in.rho_min : in.mu_ref, 2.0 * smin);
    }

    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    CKB(cudaEventRecord(e0, st));
    const int chunk = std::max(1, in.check_every);
    long long it = 0, float_iters = 0;
    bool promoted = false;
    int ok = RVE_OK;
    if (bulk) {
        pf.factor(0, 0.0);
        k_binit<D, float><<<eg, kBT, 0, st>>>(pf.a);
        launches += 2;
        // switch to FP64 once both residuals are within a few hundred float roundings of
        // their scale (sqrt(min kappa) for |D p| of a unit p; times rho / mu_ref for r_d),
        // or after 200 iterations without a 1 % gain
        double best = 1e300;
        long long best_it = 0;
        while (it < in.max_iter) {
            const long long m = std::min<long long>(chunk, in.max_iter - it);
            const long long l = pf.chunk(it, m, chunk);
            if (l < 0 || !read_ctrl()) {
                ok = RVE_E_CUDA;
                break;
            }
            launches += l;
            it += m;
            const double scale = sqrt(fmax(hc->pole / hc->rho, 0.0));
            const double eps = 256.0 * 5.96e-8 * scale;
            const double res = fmax(hc->rp, hc->rd * in.mu_ref / hc->rho);
            if (res < 0.99 * best) {
                best = res;
                best_it = it;
            }
            if (hc->stop == 3) break;
            if (hc->stop == 1 || (hc->rp <= eps && hc->rd <= eps * hc->rho / in.mu_ref) || it - best_it >= 200) {
                promoted = in.promote;  // RVE_FP32 ends here
                break;
            }
        }
        float_iters = it;
        pf.drop();
        if (promoted && (ok != RVE_OK || hc->stop == 3 || it >= in.max_iter)) promoted = false;
        if (promoted) {
            // promote: p_k and g to double, the double factor and Step 1' (forced redo)
            const long long k = hc->k;
            k_bpromote<D><<<eg, kBT, 0, st>>>((k & 1) ? pf.a.P1 : pf.a.P0, pf.a.g, (k & 1) ? pd.a.P1 : pd.a.P0,
                                              pd.a.g, (int)V);
            const int one = 1, zero = 0;
            CKB(cudaMemcpyAsync(&dctrl->stop, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
            CKB(cudaMemcpyAsync(&dctrl->rho_changed, &one, sizeof(int), cudaMemcpyHostToDevice, st));
            pd.factor(1, 0.0);
            k_bredo<D, double><<<eg, kBT, 0, st>>>(pd.a, (k & 1) ? pd.a.P1 : pd.a.P0);
            launches += 3;
            hc->stop = 0;
        }
    }
    if (ok == RVE_OK && (!bulk || promoted)) {
        if (!bulk) {
            k_binit<D, double><<<eg, kBT, 0, st>>>(pd.a);
            launches += 1;
        }
        while (it < in.max_iter) {
            const long long m = std::min<long long>(chunk, in.max_iter - it);
            const long long l = pd.chunk(it, m, chunk);
            if (l < 0 || !read_ctrl()) {
                ok = RVE_E_CUDA;
                break;
            }
            launches += l;
            it += m;
            if (hc->stop) break;
        }
        pd.drop();
    }
    if (ok != RVE_OK) return ok;
    CKB(cudaEventRecord(e1, st));
    const long long k = hc->k;
    const bool fin_float = bulk && !promoted;
    if (fin_float) {
        float2* P = (k & 1) ? pf.a.P1 : pf.a.P0;
        k_brayleigh<D, float><<<eg, kBT, 0, st>>>(pf.a, P, d_rq);
        if (in.p_out) {
            std::vector<float> pfh(2 * (size_t)D * V);
            CKB(cudaMemcpyAsync(pfh.data(), P, pfh.size() * 4, cudaMemcpyDeviceToHost, st));
            CKB(cudaStreamSynchronize(st));
            for (size_t i = 0; i < pfh.size(); ++i) in.p_out[i] = pfh[i];
        }
    } else {
        double2* P = (k & 1) ? pd.a.P1 : pd.a.P0;
        k_brayleigh<D, double><<<eg, kBT, 0, st>>>(pd.a, P, d_rq);
        if (in.p_out) CKB(cudaMemcpyAsync(in.p_out, P, 16 * (size_t)D * V, cudaMemcpyDeviceToHost, st));
    }
    launches += 1;
    double rq = 0.0;
    CKB(cudaMemcpyAsync(&rq, d_rq, 8, cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    res->iterations = (int)k;
    res->float_iterations = (int)std::min<long long>(float_iters, k);
    res->converged = hc->stop == 1;
    res->beta = hc->sigma;
    res->rayleigh = rq;
    res->r_p = hc->rp;
    res->r_d = hc->rd;
    res->time_ms = (double)ms;
    res->launches = launches;
    res->fail = hc->fail;
    res->rho = hc->rho;
    if (in.hist_out && k > 0)
        CKB(cudaMemcpy(in.hist_out, pd.a.hist, 8 * 4 * (size_t)std::min<long long>(k, in.max_iter),
                       cudaMemcpyDeviceToHost));
#undef CKB
    if (hc->stop == 3) return RVE_E_NUMERICAL;
    return res->converged ? RVE_OK : RVE_E_NOT_CONVERGED;
}

}  // namespace

int bloch_run(BlochWork** w, const BlochArgs& in, BlochResult* res) {
    if (!*w) *w = new (std::nothrow) BlochWork();
    if (!*w) return RVE_E_OOM;
    memset(res, 0, sizeof(*res));
    return in.dim == 3 ? run<3>(*w, in, res) : run<2>(*w, in, res);
}

void bloch_free(BlochWork* w) {
    if (!w) return;
    if (w->base) cudaFree(w->base);
    if (w->hctrl) cudaFreeHost(w->hctrl);
    delete w;
}

}  // namespace admm
