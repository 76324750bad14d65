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
// Fields are complex double (double2), component-major (c * V + v), x fastest.
// The complex FFTs are this file's own: one block per tile of lines along an axis,
// the line in shared memory, Stockham radix-4/2/3 passes.
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

struct BArgs {
    int n, V;
    double half_n, tol, inv_mu_ref;
    int adaptive;          // Section 2.1's residual balancing of rho
    double kappa, tau, rho_floor;
    double c[3], s[3];     // cos, sin of th_j, times 1/(2h)
    const double* sym;     // s_j(m) at sym[j * n + m]
    double2 *P0, *P1, *B, *G, *g, *Q;
    double *Lf, *Linv, *W, *part, *hist;
    BCtrl* ctrl;
    int max_hist;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

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

// (D X)_ij at v from the neighbours of X (d complex components).
template <int D>
__device__ __forceinline__ void bloch_grad(const double2* __restrict__ X, const BArgs& a, const int* up,
                                           const int* dn, double2* out) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const double2 u = X[(size_t)i * a.V + up[j]], w = X[(size_t)i * a.V + dn[j]];
            const double c = a.c[j], s = a.s[j];
            out[i * D + j] = make_double2((u.x * c - u.y * s) - (w.x * c + w.y * s),
                                          (u.x * s + u.y * c) - (w.y * c - w.x * s));
        }
}

// (D X)_ij at v for one (i, j).
__device__ __forceinline__ double2 bloch_grad1(const double2* __restrict__ X, const BArgs& a, int i, int j, int up,
                                               int dn) {
    const double2 u = X[(size_t)i * a.V + up], w = X[(size_t)i * a.V + dn];
    const double c = a.c[j], s = a.s[j];
    return make_double2((u.x * c - u.y * s) - (w.x * c + w.y * s), (u.x * s + u.y * c) - (w.y * c - w.x * s));
}

// Packed lower-triangle index.
__host__ __device__ constexpr int tri(int p, int q) { return p * (p + 1) / 2 + q; }

// (L + rho I) x = b by the stored factor (real L, complex x and b).
template <int NN>
__device__ __forceinline__ void fsolve(const BArgs& a, int v, const double2* b, double2* x) {
    double2 y[NN];
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        double2 s = b[p];
#pragma unroll
        for (int r = 0; r < p; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x -= l * y[r].x;
            s.y -= l * y[r].y;
        }
        y[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
#pragma unroll
    for (int p = NN - 1; p >= 0; --p) {
        double2 s = y[p];
#pragma unroll
        for (int r = p + 1; r < NN; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x -= l * x[r].x;
            s.y -= l * x[r].y;
        }
        x[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
}

// (L + rho I) x = b in place (forward substitution into b, then backward).
template <int NN>
__device__ __forceinline__ void fsolve_inplace(const BArgs& a, int v, double2* b) {
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        double2 s = b[p];
#pragma unroll
        for (int r = 0; r < p; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x -= l * b[r].x;
            s.y -= l * b[r].y;
        }
        b[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
#pragma unroll
    for (int p = NN - 1; p >= 0; --p) {
        double2 s = b[p];
#pragma unroll
        for (int r = p + 1; r < NN; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x -= l * b[r].x;
            s.y -= l * b[r].y;
        }
        b[p] = cscale(s, __ldg(a.Linv + (size_t)p * a.V + v));
    }
}

// y = (L + rho I) x = F (F^T x) with the stored factor F.
template <int NN>
__device__ __forceinline__ void fapply(const BArgs& a, int v, const double2* x, double2* y) {
    double2 t[NN];
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = p; r < NN; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(r, p) * a.V + v);
            s.x += l * x[r].x;
            s.y += l * x[r].y;
        }
        t[p] = s;
    }
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = 0; r <= p; ++r) {
            const double l = __ldg(a.Lf + (size_t)tri(p, r) * a.V + v);
            s.x += l * t[r].x;
            s.y += l * t[r].y;
        }
        y[p] = s;
    }
}

// kappa(m) = sum_j s_j(m_j)^2 with explicit roundings (no contraction), so that every
// kernel forms the same value.
template <int D>
__device__ __forceinline__ double kappa_of(const BArgs& a, int v) {
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

// ------------------------------------------------------------------ kernels
// Every kernel takes rho from the control block: the adaptive rule changes it between
// iterations.

// L + rho I = W_FF(F) + rho I per voxel (compressible neo-Hookean, Section 4.1, or
// isotropic linear elasticity), Cholesky-factored in double.
// mode 0: factor with ctrl->rho; mode 1: the same, only when rho changed (redo after the
// rule); mode 2: no factor stored, only the positive-definiteness test of L + shift I
// (fail bit 1), for the floor's bisection.
template <int D, int MODEL, typename TF>
__global__ void __launch_bounds__(kBT) k_bfactor(BArgs a, const TF* __restrict__ F, const uint8_t* __restrict__ phase,
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
                    if (mode != 2) a.Linv[(size_t)p * a.V + v] = ok ? 1.0 / d : 0.0;
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
        for (int p = 0; p < NN * (NN + 1) / 2; ++p) a.Lf[(size_t)p * a.V + v] = H[p];
    }
}

// Start: g_0 = L D p_0, then Step 1' of the first iteration (G, Q).
template <int D>
__global__ void __launch_bounds__(kBT) k_binit(BArgs a) {
    constexpr int NN = D * D;
    const double rho = a.ctrl->rho, inv_rho = 1.0 / rho;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        double2 Dp[NN], y[NN], rhs[NN], G[NN];
        bloch_grad<D>(a.P0, a, up, dn, Dp);
        fapply<NN>(a, v, Dp, y);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            const double2 g0 = csub(y[p], cscale(Dp[p], rho));
            y[p] = g0;
            rhs[p] = cadd(g0, cscale(Dp[p], rho));
        }
        fsolve<NN>(a, v, rhs, G);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.g[(size_t)p * a.V + v] = y[p];
            a.G[(size_t)p * a.V + v] = G[p];
            a.Q[(size_t)p * a.V + v] = make_double2(G[p].x - y[p].x * inv_rho, G[p].y - y[p].y * inv_rho);
        }
    }
}

// b = D^* Q: (D^* Q)_i = sum_j (Q_ij(x - h e_j) e^{-i th_j} - Q_ij(x + h e_j) e^{i th_j}) / (2h).
template <int D>
__global__ void __launch_bounds__(kBT) k_bdiv(BArgs a) {
    if (a.ctrl->stop) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->rho_changed = 0;  // the redo (if any) has run
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const double2 w = a.Q[(size_t)(i * D + j) * a.V + dn[j]], u = a.Q[(size_t)(i * D + j) * a.V + up[j]];
                const double c = a.c[j], s = a.s[j];
                re += (w.x * c + w.y * s) - (u.x * c - u.y * s);
                im += (w.y * c - w.x * s) - (u.x * s + u.y * c);
            }
            a.B[(size_t)i * a.V + v] = make_double2(re, im);
        }
    }
}

// In-place complex FFT of the d components of B along one axis.  A block takes a tile
// of tl lines (consecutive rows for the x axis, consecutive x (or x-y plane
// positions) for the others, so that loads coalesce), holds it in shared memory and
// runs Stockham passes of radix 4, 2 and 3 (tw[t] = exp(-2 pi i t / n)).
template <int D, int AXIS, bool INV>
__global__ void __launch_bounds__(kBT) k_bfft(BArgs a, const double2* __restrict__ tw, FftPlanB pl) {
    if (a.ctrl->stop) return;
    extern __shared__ double2 bsm[];
    const int n = pl.n, tl = pl.tl;
    const int nl = a.V / n;
    const int ntile = (nl + tl - 1) / tl;
    double2* s0 = bsm;
    double2* s1 = bsm + tl * n;
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
        double2* base = a.B + (size_t)comp * a.V;
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
        double2* in = s0;
        double2* out = s1;
        int ns = 1;
        for (int ps = 0; ps < pl.npass; ++ps) {
            const int R = pl.radix[ps], m = n / R, tws = n / (ns * R);
            for (int t = threadIdx.x; t < tl * m; t += kBT) {
                const int l = t / m, j = t - l * m, kk = j % ns;
                const double2* li = in + l * n;
                double2* lo = out + l * n;
                const int o = (j - kk) * R + kk;
                double2 x0 = li[j], x1 = li[j + m];
                if (kk) {
                    double2 w = tw[kk * tws];
                    if (INV) w.y = -w.y;
                    x1 = cmul(x1, w);
                }
                if (R == 2) {
                    lo[o] = cadd(x0, x1);
                    lo[o + ns] = csub(x0, x1);
                } else if (R == 3) {
                    double2 x2 = li[j + 2 * m];
                    if (kk) {
                        double2 w = tw[2 * kk * tws];
                        if (INV) w.y = -w.y;
                        x2 = cmul(x2, w);
                    }
                    // y1,2 = x0 - (x1 + x2)/2 -+ i sqrt(3)/2 (x1 - x2) (forward; signs swap inverse)
                    const double h3 = INV ? -0.86602540378443864676 : 0.86602540378443864676;
                    const double2 t1 = cadd(x1, x2), t2 = csub(x1, x2);
                    const double2 mid = make_double2(x0.x - 0.5 * t1.x, x0.y - 0.5 * t1.y);
                    lo[o] = cadd(x0, t1);
                    lo[o + ns] = make_double2(mid.x + h3 * t2.y, mid.y - h3 * t2.x);
                    lo[o + 2 * ns] = make_double2(mid.x - h3 * t2.y, mid.y + h3 * t2.x);
                } else {
                    double2 x2 = li[j + 2 * m], x3 = li[j + 3 * m];
                    if (kk) {
                        double2 w2 = tw[2 * kk * tws], w3 = tw[3 * kk * tws];
                        if (INV) {
                            w2.y = -w2.y;
                            w3.y = -w3.y;
                        }
                        x2 = cmul(x2, w2);
                        x3 = cmul(x3, w3);
                    }
                    // y0 = a0+a1+a2+a3, y2 = a0-a1+a2-a3, y1,3 = (a0-a2) -+ i (a1-a3) (forward)
                    const double2 e = cadd(x0, x2), f = csub(x0, x2), g2 = cadd(x1, x3), h = csub(x1, x3);
                    lo[o] = cadd(e, g2);
                    lo[o + 2 * ns] = csub(e, g2);
                    if (!INV) {
                        lo[o + ns] = make_double2(f.x + h.y, f.y - h.x);
                        lo[o + 3 * ns] = make_double2(f.x - h.y, f.y + h.x);
                    } else {
                        lo[o + ns] = make_double2(f.x - h.y, f.y + h.x);
                        lo[o + 3 * ns] = make_double2(f.x + h.y, f.y - h.x);
                    }
                }
            }
            __syncthreads();
            double2* sw = in;
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

template <int D>
__global__ void __launch_bounds__(kBT) k_bweights(BArgs a) {
    if (a.ctrl->stop) return;
    double ws = 0.0, km = 1e300, wm = 0.0;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        double w = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double2 b = a.B[(size_t)i * a.V + v];
            w += b.x * b.x + b.y * b.y;
        }
        a.W[v] = w;
        ws += w;
        kw_merge(km, wm, kappa_of<D>(a, v), w);
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
template <int D>
__global__ void __launch_bounds__(kBT) k_broot(BArgs a, int last) {
    const BCtrl* cc = a.ctrl;
    if (cc->stop || cc->root_done) return;
    const double sig = cc->sigma, rho = cc->rho, r2 = rho * rho;
    double v2[2] = {0.0, 0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        const double inv = 1.0 / __dsub_rn(__dmul_rn(rho, kappa_of<D>(a, v)), sig);
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
template <int D>
__global__ void __launch_bounds__(kBT) k_bphat(BArgs a) {
    if (a.ctrl->stop) return;
    const double sig = a.ctrl->sigma, rho = a.ctrl->rho, Vd = (double)a.V;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        const double den = __dsub_rn(__dmul_rn(rho, kappa_of<D>(a, v)), sig);
        const double f = rho / (den * Vd);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const double2 b = a.B[(size_t)i * a.V + v];
            a.B[(size_t)i * a.V + v] = make_double2(b.x * f, b.y * f);
        }
    }
}

// Steps 3' and 4' of iteration i (p_i in B, p_{i-1} in Pold, G_i, g_{i-1}) fused with
// Step 1' of iteration i + 1 (G_{i+1}, Q); p_i is copied to Pnew.  The last block
// finishes the residuals, records them and sets the stop flag.
template <int D>
__global__ void __launch_bounds__(kBT, 2) k_blocal(BArgs a, const double2* __restrict__ Pold, double2* __restrict__ Pnew) {
    constexpr int NN = D * D;
    if (a.ctrl->stop) return;
    const double rho = a.ctrl->rho, inv_rho = 1.0 / rho;
    double v2[2] = {0.0, 0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        double2 x[NN], gn[NN];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int p = i * D + j;
                const double2 Dn = bloch_grad1(a.B, a, i, j, up[j], dn[j]);
                const double2 Do = bloch_grad1(Pold, a, i, j, up[j], dn[j]);
                const double2 e = csub(Dn, a.G[(size_t)p * a.V + v]), dd = csub(Dn, Do);
                v2[0] += e.x * e.x + e.y * e.y;
                v2[1] += dd.x * dd.x + dd.y * dd.y;
                gn[p] = cadd(a.g[(size_t)p * a.V + v], cscale(e, rho));  // Step 3'
                x[p] = cadd(gn[p], cscale(Dn, rho));
            }
        fsolve_inplace<NN>(a, v, x);  // Step 1' of the next iteration
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.g[(size_t)p * a.V + v] = gn[p];
            a.G[(size_t)p * a.V + v] = x[p];
            a.Q[(size_t)p * a.V + v] = make_double2(x[p].x - gn[p].x * inv_rho, x[p].y - gn[p].y * inv_rho);
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
template <int D>
__global__ void __launch_bounds__(kBT) k_bredo(BArgs a, const double2* __restrict__ P) {
    constexpr int NN = D * D;
    if (a.ctrl->stop || !a.ctrl->rho_changed) return;
    const double rho = a.ctrl->rho, inv_rho = 1.0 / rho;
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        double2 x[NN], gv[NN];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int p = i * D + j;
                gv[p] = a.g[(size_t)p * a.V + v];
                x[p] = cadd(gv[p], cscale(bloch_grad1(P, a, i, j, up[j], dn[j]), rho));
            }
        fsolve_inplace<NN>(a, v, x);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            a.G[(size_t)p * a.V + v] = x[p];
            a.Q[(size_t)p * a.V + v] = make_double2(x[p].x - gv[p].x * inv_rho, x[p].y - gv[p].y * inv_rho);
        }
    }
}

// <D p, L D p> = mean over voxels of |F^T Dp|^2 - rho |Dp|^2 (F the stored factor).
template <int D>
__global__ void __launch_bounds__(kBT) k_brayleigh(BArgs a, const double2* __restrict__ P, double* out) {
    constexpr int NN = D * D;
    const double rho = a.ctrl->rho;
    double v1[1] = {0.0};
    for (int v = blockIdx.x * kBT + threadIdx.x; v < a.V; v += gridDim.x * kBT) {
        int up[3], dn[3];
        bneighbours<D>(v, a.n, up, dn);
        double2 Dp[NN], y[NN];
        bloch_grad<D>(P, a, up, dn, Dp);
        fapply<NN>(a, v, Dp, y);
#pragma unroll
        for (int p = 0; p < NN; ++p) v1[0] += (Dp[p].x * y[p].x + Dp[p].y * y[p].y) - rho * (Dp[p].x * Dp[p].x + Dp[p].y * Dp[p].y);
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

template <int D>
cudaError_t set_fft_attrs(size_t smem) {
    static size_t done[2] = {0, 0};
    if (done[D - 2] >= smem) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const int b = (int)smem;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 0, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bfft<D, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (D == 3) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bfft<D, D - 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bfft<D, D - 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
    if (e == cudaSuccess) done[D - 2] = smem;
    return e;
}

template <int D, bool INV>
void fft_all(const BArgs& a, const double2* tw, const FftPlanB& pl, size_t smem, int fg, cudaStream_t st) {
    k_bfft<D, 0, INV><<<fg, kBT, smem, st>>>(a, tw, pl);
    k_bfft<D, 1, INV><<<fg, kBT, smem, st>>>(a, tw, pl);
    if (D == 3) k_bfft<D, D - 1, INV><<<fg, kBT, smem, st>>>(a, tw, pl);
}

template <int D>
int run(BlochWork* w, const BlochArgs& in, BlochResult* res) {
    constexpr int NN = D * D;
    const int n = in.n;
    const long long V = in.V;
    cudaStream_t st = in.stream;
    // workspace layout
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 255) / 256 * 256;
        return o;
    };
    const size_t oP0 = take(16 * D * V), oP1 = take(16 * D * V), oB = take(16 * D * V);
    const size_t oG = take(16 * NN * V), og = take(16 * NN * V), oQ = take(16 * NN * V);
    const size_t oL = take(8 * (size_t)(NN * (NN + 1) / 2) * V), oLi = take(8 * NN * V), oW = take(8 * V);
    const size_t opart = take(8 * 4 * kBlochBlocks), ohist = take(8 * 4 * (size_t)in.max_iter);
    const size_t osym = take(8 * 3 * n), otw = take(16 * n), octrl = take(sizeof(BCtrl)), orq = take(8);
    if (w->bytes < off) {
        if (w->base) cudaFree(w->base);
        w->base = nullptr;
        w->bytes = 0;
        if (cudaMalloc((void**)&w->base, off) != cudaSuccess) return RVE_E_OOM;
        w->bytes = off;
    }
    if (!w->hctrl && cudaMallocHost(&w->hctrl, sizeof(BCtrl) + 64) != cudaSuccess) return RVE_E_OOM;
    unsigned char* b = w->base;
    BArgs a{};
    a.n = n;
    a.V = (int)V;
    a.half_n = 0.5 * n;
    a.tol = in.tol;
    a.inv_mu_ref = 1.0 / in.mu_ref;
    a.adaptive = in.adaptive ? 1 : 0;
    a.kappa = in.rho_kappa;
    a.tau = in.rho_tau;
    a.rho_floor = 0.0;
    for (int j = 0; j < 3; ++j) {
        const double th = j < D ? 2.0 * kPi / ((double)in.k[j] * n) : 0.0;
        a.c[j] = a.half_n * cos(th);
        a.s[j] = a.half_n * sin(th);
    }
    a.P0 = (double2*)(b + oP0);
    a.P1 = (double2*)(b + oP1);
    a.B = (double2*)(b + oB);
    a.G = (double2*)(b + oG);
    a.g = (double2*)(b + og);
    a.Q = (double2*)(b + oQ);
    a.Lf = (double*)(b + oL);
    a.Linv = (double*)(b + oLi);
    a.W = (double*)(b + oW);
    a.part = (double*)(b + opart);
    a.hist = (double*)(b + ohist);
    a.sym = (const double*)(b + osym);
    a.ctrl = (BCtrl*)(b + octrl);
    a.max_hist = in.max_iter;
    double* d_rq = (double*)(b + orq);
    double2* tw = (double2*)(b + otw);

    // host-side tables and the normalised start
    std::vector<double> sym(3 * (size_t)n, 0.0);
    for (int j = 0; j < D; ++j)
        for (int m = 0; m < n; ++m) sym[(size_t)j * n + m] = n * sin(2.0 * kPi * (m + 1.0 / in.k[j]) / n);
    std::vector<double2> twh(n);
    for (int t = 0; t < n; ++t) twh[t] = make_double2(cos(2.0 * kPi * t / n), -sin(2.0 * kPi * t / n));
    double nrm = 0.0;
    for (size_t i = 0; i < 2 * (size_t)D * V; ++i) nrm += in.p0[i] * in.p0[i];
    nrm = sqrt(nrm / (double)V);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return RVE_E_INVALID_ARG;
    std::vector<double> p0((size_t)2 * D * V);
    for (size_t i = 0; i < p0.size(); ++i) p0[i] = in.p0[i] / nrm;
    BCtrl c0{};
    c0.sigma = NAN;
    c0.rho = in.rho;
#define CKB(x)                                  \
    do {                                        \
        if ((x) != cudaSuccess) return RVE_E_CUDA; \
    } while (0)
    CKB(cudaMemcpyAsync((void*)a.sym, sym.data(), sym.size() * 8, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(tw, twh.data(), twh.size() * 16, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(a.P0, p0.data(), p0.size() * 8, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(a.ctrl, &c0, sizeof(BCtrl), cudaMemcpyHostToDevice, st));
    const FftPlanB pl = make_plan(n);
    const size_t smem = (size_t)2 * pl.tl * n * sizeof(double2);
    CKB(set_fft_attrs<D>(smem));
    const int eg = grid_for(V);
    const int ntiles = (int)((V / n + pl.tl - 1) / pl.tl) * D;
    const int fg = std::min(ntiles, 152 * 3);
    long long launches = 0;
    auto factor = [&](int mode, double shift) {
        if (in.model == kNeoHooke) {
            if (in.F_fp64)
                k_bfactor<D, kNeoHooke, double><<<eg, kBT, 0, st>>>(a, (const double*)in.F, in.phase, in.mat, in.nparam,
                                                                    mode, shift);
            else
                k_bfactor<D, kNeoHooke, float><<<eg, kBT, 0, st>>>(a, (const float*)in.F, in.phase, in.mat, in.nparam,
                                                                   mode, shift);
        } else {
            if (in.F_fp64)
                k_bfactor<D, kLinear, double><<<eg, kBT, 0, st>>>(a, (const double*)in.F, in.phase, in.mat, in.nparam,
                                                                  mode, shift);
            else
                k_bfactor<D, kLinear, float><<<eg, kBT, 0, st>>>(a, (const float*)in.F, in.phase, in.mat, in.nparam,
                                                                 mode, shift);
        }
    };
    BCtrl* hc = (BCtrl*)w->hctrl;
    factor(0, 0.0);
    launches += 1;
    CKB(cudaMemcpyAsync(hc, a.ctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    CKB(cudaGetLastError());
    if (hc->fail & 1) return RVE_E_NUMERICAL;
    if (a.adaptive) {
        // floor of the rule: max(rho_min or mu_ref, 2 s*), s* the smallest shift with
        // L + s* I positive definite everywhere (bisection on [0, rho], to 2^-16 rho)
        auto pd = [&](double sft) -> int {
            if (cudaMemsetAsync(&a.ctrl->fail, 0, sizeof(int), st) != cudaSuccess) return -1;
            factor(2, sft);
            launches += 1;
            if (cudaMemcpyAsync(hc, a.ctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return -1;
            return (hc->fail & 1) ? 0 : 1;
        };
        double smin = 0.0;
        int r0 = pd(0.0);
        if (r0 < 0) return RVE_E_CUDA;
        if (!r0) {
            double lo = 0.0, hi = in.rho;
            for (int b = 0; b < 16; ++b) {
                const double mid = 0.5 * (lo + hi);
                const int r = pd(mid);
                if (r < 0) return RVE_E_CUDA;
                if (r) hi = mid;
                else lo = mid;
            }
            smin = hi;
        }
        CKB(cudaMemsetAsync(&a.ctrl->fail, 0, sizeof(int), st));
        a.rho_floor = std::max(in.rho_min > 0.0 ? in.rho_min : in.mu_ref, 2.0 * smin);
    }
    k_binit<D><<<eg, kBT, 0, st>>>(a);
    launches += 1;

    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    CKB(cudaEventRecord(e0, st));
    auto iteration = [&](long long i) {  // iteration i reads p_{i-1} and writes p_i
        double2* Pold = ((i - 1) & 1) ? a.P1 : a.P0;
        double2* Pnew = (i & 1) ? a.P1 : a.P0;
        const int passes = i == 1 ? kRootPasses0 : (i == 2 ? kRootPasses1 : kRootPasses);
        k_bdiv<D><<<eg, kBT, 0, st>>>(a);
        fft_all<D, false>(a, tw, pl, smem, fg, st);
        k_bweights<D><<<eg, kBT, 0, st>>>(a);
        for (int r = 0; r < passes; ++r) k_broot<D><<<eg, kBT, 0, st>>>(a, r == passes - 1);
        k_bphat<D><<<eg, kBT, 0, st>>>(a);
        fft_all<D, true>(a, tw, pl, smem, fg, st);
        k_blocal<D><<<eg, kBT, 0, st>>>(a, Pold, Pnew);
        if (a.adaptive) {  // after a change of rho: new factor, Step 1' again
            factor(1, 0.0);
            k_bredo<D><<<eg, kBT, 0, st>>>(a, Pnew);
        }
        return 4 + 2 * D + passes + (a.adaptive ? 2 : 0);
    };
    // The first chunk runs as plain launches (its first iterations take more root
    // passes); later full chunks replay a graph per starting parity of p.
    long long it = 0;
    const int chunk = std::max(1, in.check_every);
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int per_chunk = 0;
    auto drop_graphs = [&]() {
        for (auto& g : graph)
            if (g) cudaGraphExecDestroy(g);
    };
    while (it < in.max_iter) {
        const long long m = std::min<long long>(chunk, in.max_iter - it);
        if (it >= 2 && m == chunk) {
            const int par = (int)(it & 1);
            if (!graph[par]) {
                cudaGraph_t g = nullptr;
                per_chunk = 0;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                    drop_graphs();
                    return RVE_E_CUDA;
                }
                for (long long q = 0; q < m; ++q) per_chunk += iteration(it + q + 1);
                const cudaError_t ec = cudaStreamEndCapture(st, &g);
                const cudaError_t ei = ec == cudaSuccess ? cudaGraphInstantiate(&graph[par], g, 0) : ec;
                if (g) cudaGraphDestroy(g);
                if (ei != cudaSuccess) {
                    drop_graphs();
                    return RVE_E_CUDA;
                }
            }
            if (cudaGraphLaunch(graph[par], st) != cudaSuccess) {
                drop_graphs();
                return RVE_E_CUDA;
            }
            launches += per_chunk;
        } else {
            for (long long q = 0; q < m; ++q) launches += iteration(it + q + 1);
        }
        if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(hc, a.ctrl, sizeof(BCtrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            drop_graphs();
            return RVE_E_CUDA;
        }
        it += m;
        if (hc->stop) break;
    }
    drop_graphs();
    CKB(cudaEventRecord(e1, st));
    const long long k = hc->k;
    double2* Pfin = (k & 1) ? a.P1 : a.P0;
    k_brayleigh<D><<<eg, kBT, 0, st>>>(a, Pfin, d_rq);
    launches += 1;
    double rq = 0.0;
    CKB(cudaMemcpyAsync(&rq, d_rq, 8, cudaMemcpyDeviceToHost, st));
    if (in.p_out) CKB(cudaMemcpyAsync(in.p_out, Pfin, 16 * (size_t)D * V, cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    res->iterations = (int)k;
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
        CKB(cudaMemcpy(in.hist_out, a.hist, 8 * 4 * (size_t)std::min<long long>(k, in.max_iter),
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
