// Local (pointwise) kernels of the ADMM iteration, Zhou & Bhattacharya Section 2.1:
//   Step 1 (eq. eq)      F_{i+1} = argmin_F W(F;x) - Lambda_i : F + rho/2 |F - G_i|^2
//   Step 3 (eq. update)  Lambda_{i+1} = Lambda_i + rho (G_{i+1} - F_{i+1})
//   Step 4 (eq. check)   r_p = ||G_{i+1} - F_{i+1}||,  r_d = rho/mu ||G_{i+1} - G_i||
// with G = Fbar + D u~ and D the central-difference gradient of Section 2.3.
//
// One fused kernel per iteration finishes Steps 3-4 of iteration i and runs Step 1
// of iteration i+1 at each voxel, so F, Lambda and u~ are read once and F, Lambda
// written once per iteration.  One thread owns one voxel; the 3x3 (2x2) algebra,
// the 9x9 (4x4) Newton Hessian and its Cholesky factor live in registers.
// Residual sums are accumulated in double whatever the field precision, reduced
// per block with warp shuffles and finished by the last block in a fixed order,
// so the result does not depend on block scheduling.
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "rve_internal.cuh"

namespace admm {
namespace {

// ------------------------------------------------------------------ small dense algebra

template <typename T, int D>
__device__ __forceinline__ T det_cof(const T* F, T* K) {
    if constexpr (D == 2) {
        K[0] = F[3];
        K[1] = -F[2];
        K[2] = -F[1];
        K[3] = F[0];
        return F[0] * F[3] - F[1] * F[2];
    } else {
        K[0] = F[4] * F[8] - F[5] * F[7];
        K[1] = F[5] * F[6] - F[3] * F[8];
        K[2] = F[3] * F[7] - F[4] * F[6];
        K[3] = F[2] * F[7] - F[1] * F[8];
        K[4] = F[0] * F[8] - F[2] * F[6];
        K[5] = F[1] * F[6] - F[0] * F[7];
        K[6] = F[1] * F[5] - F[2] * F[4];
        K[7] = F[2] * F[3] - F[0] * F[5];
        K[8] = F[0] * F[4] - F[1] * F[3];
        return F[0] * K[0] + F[1] * K[1] + F[2] * K[2];
    }
}

template <typename T, int D>
__device__ __forceinline__ T det(const T* F) {
    if constexpr (D == 2) {
        return F[0] * F[3] - F[1] * F[2];
    } else {
        return F[0] * (F[4] * F[8] - F[5] * F[7]) + F[1] * (F[5] * F[6] - F[3] * F[8]) +
               F[2] * (F[3] * F[7] - F[4] * F[6]);
    }
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

// ------------------------------------------------------------------ double-word arithmetic
// A double-word number is the unevaluated sum hi + lo of two floats with |lo| <=
// ulp(hi) / 2: about 48 significant bits, from FP32 instructions only.  GB300
// executes FP32 at 64 times its FP64 rate, so the double polish keeps its state as
// pairs of floats and forms its linearisation offsets in this arithmetic
// (polish_voxel_dev).  Error-free transformations: two_sum (Knuth), fast_two_sum
// (Dekker, needs |a| >= |b| or a = 0), two_prod with an FMA.
// The sum, product and quotient are the double-word algorithms analysed by Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017 (relative errors of a few u^2,
// u = 2^-24: sum of two double-words 3u^2, double-word times float 2u^2, product
// 5u^2, quotient 15u^2).  The _rn intrinsics stop the compiler from contracting or
// reassociating the operations these rely on.
struct dw {
    float hi, lo;
};
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dw two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dw{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dw two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dw{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dw dw_neg(dw x) { return dw{-x.hi, -x.lo}; }
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = two_sum(x.hi, y.hi);
    const dw t = two_sum(x.lo, y.lo);
    const dw v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ dw dw_add_f(dw x, float y) {
    const dw s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    const dw c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const dw c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, __fmaf_rn(x.lo, y.hi, t)));
}
__device__ __forceinline__ dw dw_div(dw x, dw y) {
    const float th = __fdiv_rn(x.hi, y.hi);
    const dw r = dw_mul_f(y, th);
    const float d = __fadd_rn(__fsub_rn(x.hi, r.hi), __fsub_rn(x.lo, r.lo));
    return fast_two_sum(th, __fdiv_rn(d, y.hi));
}
// exact split of a double into a double-word (|d| within the float range), and back
__device__ __forceinline__ dw dw_from(double d) {
    const float hi = (float)d;
    return dw{hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ double dw_to(dw x) { return (double)x.hi + (double)x.lo; }

// Cholesky factor of a symmetric positive definite H in packed lower storage
// (row p, column q <= p at p(p+1)/2 + q), in place, with the reciprocal pivots in
// inv.  Returns false when a pivot is not positive.
template <typename T, int N>
__device__ __forceinline__ bool chol_factor(T* H, T* inv) {
#pragma unroll
    for (int p = 0; p < N; ++p) {
#pragma unroll
        for (int q = 0; q <= p; ++q) {
            T s = H[p * (p + 1) / 2 + q];
#pragma unroll
            for (int r = 0; r < q; ++r) s -= H[p * (p + 1) / 2 + r] * H[q * (q + 1) / 2 + r];
            if (p == q) {
                if (!(s > T(0))) return false;
                const T is = rsqrt_t(s);
                inv[p] = is;
                H[p * (p + 1) / 2 + p] = s * is;
            } else {
                H[p * (p + 1) / 2 + q] = s * inv[q];
            }
        }
    }
    return true;
}

// x = -H^{-1} g from the factor of chol_factor (forward, then back substitution).
template <typename T, int N>
__device__ __forceinline__ void chol_subst(const T* H, const T* inv, const T* g, T* x) {
    T y[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        T s = -g[p];
#pragma unroll
        for (int r = 0; r < p; ++r) s -= H[p * (p + 1) / 2 + r] * y[r];
        y[p] = s * inv[p];
    }
#pragma unroll
    for (int p = N - 1; p >= 0; --p) {
        T s = y[p];
#pragma unroll
        for (int r = p + 1; r < N; ++r) s -= H[r * (r + 1) / 2 + p] * x[r];
        x[p] = s * inv[p];
    }
}

// Solve H x = -g; H is overwritten by its Cholesky factor.
template <typename T, int N>
__device__ __forceinline__ bool chol_solve(T* H, const T* g, T* x) {
    T inv[N];
    if (!chol_factor<T, N>(H, inv)) return false;
    chol_subst<T, N>(H, inv, g, x);
    return true;
}

// ------------------------------------------------------------------ constitutive laws
// Each law gives, for the local objective phi(F) = W(F) + rho/2 |F|^2 - B : F
// (B = Lambda + rho G; the constant rho/2 |G|^2 is dropped):
//   grad:   g = W_F(F) + rho F - B in the field precision T, plus the auxiliary
//           values the Hessian needs (law-specific)
//   hess:   the packed Hessian W_FF + rho I, always in float (see newton())
//   phi:    the objective (line search);  stress: W_F(F)

// Compressible neo-Hookean, Section 4.1: W = mu/2 (|F|^2 - d - 2 ln J) + lam/2 (J-1)^2.
// W_F = mu F + c F^{-T}, c = lam J (J-1) - mu;
// W_FF[ij,kl] = mu d_ik d_jl + lam (2J-1) J A_ij A_kl - c A_il A_kj, A = F^{-T}.
// The auxiliary values are the cofactor matrix K = J F^{-T} and J; the gradient
// uses c / J times K, and the float side forms A = K / J itself.
template <typename T, int D>
struct NeoHooke {
    T mu, lam;
    static constexpr int NAUX = D * D + 1;
    __device__ __forceinline__ bool grad(const T* F, const T* B, T rho, T* g, T* aux) const {
        constexpr int NN = D * D;
        T* K = aux;
        const T J = det_cof<T, D>(F, K);
        aux[NN] = J;
        if (!(J > T(0))) return false;
        const T cJ = (lam * J * (J - T(1)) - mu) / J;
        const T a = mu + rho;
#pragma unroll
        for (int p = 0; p < NN; ++p) g[p] = a * F[p] + cJ * K[p] - B[p];
        return true;
    }
    __device__ __forceinline__ void hess(const float* aux, float rho, float* H) const {
        constexpr int NN = D * D;
        const float J = aux[NN];
        const float iJ = 1.f / J;
        float A[NN];
#pragma unroll
        for (int p = 0; p < NN; ++p) A[p] = aux[p] * iJ;
        const float fm = (float)mu, fl = (float)lam;
        const float c = fl * J * (J - 1.f) - fm;
        const float b = fl * (2.f * J - 1.f) * J;
        const float a = fm + rho;
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            const int i = p / D, j = p % D;
#pragma unroll
            for (int q = 0; q <= p; ++q) {
                const int k = q / D, l = q % D;
                float h = b * A[p] * A[q] - c * A[i * D + l] * A[k * D + j];
                if (p == q) h += a;
                H[p * (p + 1) / 2 + q] = h;
            }
        }
    }
    __device__ __forceinline__ T phi(const T* F, const T* B, T rho, T J) const {
        T ff = 0, bf = 0;
#pragma unroll
        for (int p = 0; p < D * D; ++p) {
            ff += F[p] * F[p];
            bf += B[p] * F[p];
        }
        return T(0.5) * mu * (ff - T(2) * log_t(J)) + T(0.5) * lam * (J - T(1)) * (J - T(1)) +
               T(0.5) * rho * ff - bf;
    }
    __device__ __forceinline__ void stress(const T* F, T* P) const {
        T A[D * D];
        const T J = det_cof<T, D>(F, A);
        const T c = (lam * J * (J - T(1)) - mu) / J;
#pragma unroll
        for (int p = 0; p < D * D; ++p) P[p] = mu * F[p] + c * A[p];
    }
    __device__ __forceinline__ T modulus() const { return mu; }
    // det(F + dF) > 0 is certain when |F^{-1} dF| < 1/2: |F^{-1} dF|_2 <= |A|_F * d * max|dF|;
    // safety_scale is |A|_F = |K|_F / J, and a step is safe when d * size * scale < 1/2
    __device__ __forceinline__ float safety_scale(const float* aux) const {
        float a2 = 0.f;
#pragma unroll
        for (int p = 0; p < D * D; ++p) a2 += aux[p] * aux[p];
        return sqrtf(a2) / aux[D * D];
    }
    __device__ __forceinline__ bool small_step_safe(const float* aux, float size) const {
        return (float)D * size * safety_scale(aux) < 0.5f;
    }
};

// Isotropic linear elasticity in H = F - I: W = mu |sym H|^2 + lam/2 (tr H)^2.
template <typename T, int D>
struct Linear {
    T mu, lam;
    static constexpr int NAUX = 1;
    __device__ __forceinline__ bool grad(const T* F, const T* B, T rho, T* g, T* aux) const {
        aux[0] = T(1);
        T tr = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) tr += F[i * D + i] - T(1);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const T hij = F[i * D + j] - (i == j ? T(1) : T(0));
                const T hji = F[j * D + i] - (i == j ? T(1) : T(0));
                g[i * D + j] = mu * (hij + hji) + (i == j ? lam * tr : T(0)) + rho * F[i * D + j] - B[i * D + j];
            }
        return true;
    }
    __device__ __forceinline__ void hess(const float* /*aux*/, float rho, float* H) const {
        const float fm = (float)mu, fl = (float)lam;
#pragma unroll
        for (int p = 0; p < D * D; ++p) {
            const int i = p / D, j = p % D;
#pragma unroll
            for (int q = 0; q <= p; ++q) {
                const int k = q / D, l = q % D;
                float h = fm * (float(i == k && j == l) + float(i == l && j == k)) + fl * float(i == j && k == l);
                if (p == q) h += rho;
                H[p * (p + 1) / 2 + q] = h;
            }
        }
    }
    __device__ __forceinline__ T phi(const T* F, const T* B, T rho, T /*J*/) const {
        T e2 = 0, tr = 0, ff = 0, bf = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) {
            tr += F[i * D + i] - T(1);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const T e = T(0.5) * (F[i * D + j] + F[j * D + i]) - (i == j ? T(1) : T(0));
                e2 += e * e;
                ff += F[i * D + j] * F[i * D + j];
                bf += B[i * D + j] * F[i * D + j];
            }
        }
        return mu * e2 + T(0.5) * lam * tr * tr + T(0.5) * rho * ff - bf;
    }
    __device__ __forceinline__ void stress(const T* F, T* P) const {
        T tr = 0;
#pragma unroll
        for (int i = 0; i < D; ++i) tr += F[i * D + i] - T(1);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
                P[i * D + j] = mu * (F[i * D + j] + F[j * D + i] - T(2) * T(i == j)) + (i == j ? lam * tr : T(0));
    }
    __device__ __forceinline__ T modulus() const { return mu; }
    // no positivity requirement on J for linear elasticity, but J > 0 is kept like
    // for the other laws: small steps from a state with J > 0 are accepted directly
    __device__ __forceinline__ float safety_scale(const float*) const { return 0.f; }
    __device__ __forceinline__ bool small_step_safe(const float*, float size) const { return size < 1e-2f; }
};

template <typename T, int D, int MODEL>
struct LawOf;
template <typename T, int D>
struct LawOf<T, D, kNeoHooke> { using type = NeoHooke<T, D>; };
template <typename T, int D>
struct LawOf<T, D, kLinear> { using type = Linear<T, D>; };

template <typename Law, typename T>
__device__ __forceinline__ Law load_law(const uint8_t* phase, const T* mat, int nparam, long long v) {
    const int ph = phase[v];
    Law m;
    m.mu = __ldg(mat + ph * nparam + 0);
    m.lam = __ldg(mat + ph * nparam + 1);
    return m;
}

template <typename T>
struct NewtonConst;
template <>
struct NewtonConst<double> { static constexpr double big = 1e-2; };
template <>
struct NewtonConst<float> { static constexpr float big = 1e-2f; };

// Damped Newton for phi at one voxel, starting from F (overwritten).
//
// The gradient, the objective and the update are evaluated in the field
// precision T; the Hessian is assembled and factored in float.  For T = float
// this is plain Newton.  For T = double it is Newton with mixed-precision
// iterative refinement: each step solves H_f dx = -g with the float factor of
// the Hessian and the double gradient, so the iteration still converges to the
// double-precision stationary point g = 0 (the float factor only slows the
// quadratic rate to a linear rate of about eps_float * cond(H) per step, which
// the tolerance test absorbs), at a fraction of the double arithmetic.
//
// Steps larger than NewtonConst::big take an Armijo backtracking line search on
// phi; every step keeps J = det F > 0.  Stops after a full step with
// max|dF| <= tol.  Returns the number of Newton steps; conv tells whether the
// test was met.
template <typename T, int D, typename Law>
__device__ __forceinline__ int newton(const Law& m, T* F, const T* B, T rho, int cap, T tol, bool& conv,
                                      T gtol = T(0), T* gnorm2 = nullptr) {
    constexpr int NN = D * D;
    constexpr int NP = NN * (NN + 1) / 2;
    constexpr int NAUX = Law::NAUX;
    conv = false;
    int it = 0;
    bool small = false;  // gtol > 0: the step test was met; stop at the next gradient
    while (it < cap || small) {
        T g[NN], aux[NAUX];
        if (!m.grad(F, B, rho, g, aux)) break;
        if (gtol > T(0)) {
            T s2 = T(0);
#pragma unroll
            for (int p = 0; p < NN; ++p) s2 += g[p] * g[p];
            *gnorm2 = s2;
            if (small || s2 <= gtol * gtol) {
                conv = true;
                break;
            }
        }
        float df[NN], gf[NN], af[NAUX];
        {
            float Hf[NP];
#pragma unroll
            for (int p = 0; p < NAUX; ++p) af[p] = (float)aux[p];
#pragma unroll
            for (int p = 0; p < NN; ++p) gf[p] = (float)g[p];
            m.hess(af, (float)rho, Hf);
            if (!chol_solve<float, NN>(Hf, gf, df)) {
                const float s = 1.f / (float)(m.modulus() + rho);
#pragma unroll
                for (int p = 0; p < NN; ++p) df[p] = -gf[p] * s;
            }
        }
        // slope and step size only steer the line search and the stopping test: float suffices
        float slope = 0.f, size = 0.f;
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            slope += gf[p] * df[p];
            size = fmaxf(size, fabsf(df[p]));
        }
        if (!(slope < 0.f)) {  // not a descent direction: steepest descent (Section 2.1's local method)
            const float s = 1.f / (float)(m.modulus() + rho);
            slope = 0.f;
            size = 0.f;
#pragma unroll
            for (int p = 0; p < NN; ++p) {
                df[p] = -gf[p] * s;
                slope += gf[p] * df[p];
                size = fmaxf(size, fabsf(df[p]));
            }
        }
        if (!(size < 1e30f)) break;  // NaN or overflow
        T t = T(1);
        if (size > (float)NewtonConst<T>::big) {
            T Ft[NN];
            const T phi0 = m.phi(F, B, rho, det<T, D>(F));
            int ls = 0;
            for (; ls < 40; ++ls) {
#pragma unroll
                for (int p = 0; p < NN; ++p) Ft[p] = F[p] + t * (T)df[p];
                const T Jt = det<T, D>(Ft);
                if (Jt > T(0) && m.phi(Ft, B, rho, Jt) <= phi0 + T(1e-4) * t * (T)slope) break;
                t *= T(0.5);
            }
            if (ls == 40) t = T(0);
        } else if (!m.small_step_safe(af, size)) {
            T Ft[NN];
            int ls = 0;
            for (; ls < 40; ++ls) {
#pragma unroll
                for (int p = 0; p < NN; ++p) Ft[p] = F[p] + t * (T)df[p];
                if (det<T, D>(Ft) > T(0)) break;
                t *= T(0.5);
            }
            if (ls == 40) t = T(0);
        }
#pragma unroll
        for (int p = 0; p < NN; ++p) F[p] += t * (T)df[p];
        ++it;
        if (t == T(1) && size <= (float)tol) {
            if (gtol > T(0)) {
                small = true;
                continue;
            }
            conv = true;
            break;
        }
        if (t == T(0)) break;
    }
    return it;
}

// ------------------------------------------------------------------ closed-form Step 1, neo-Hookean, 3D, float
// Stationarity of phi(F) = W(F) + rho/2 |F|^2 - B : F for the compressible
// neo-Hookean law is  a F + c(J) F^{-T} = B,  a = mu + rho, c(J) = lam J (J - 1) - mu.
// With F = U diag(s) V^T (U, V rotations) also F^{-T} = U diag(1/s) V^T, so B has
// F's singular vectors and singular values b_i = a s_i + c / s_i: each s_i is a root
// of a s^2 - b_i s + c = 0.  The minimiser takes the larger root,
//   s_i = (b_i + q_i) / (2a),   q_i = sqrt(x_i - k),   x_i = b_i^2,   k = 4 a c,
// and the local problem becomes one scalar equation in J:  s_1 s_2 s_3 = J.  For
// J > 1/2, c grows with J and every s_i falls (ds_i/dc = -1/q_i), so there is at
// most one root; it is found by Newton's method on f(J) = s_1 s_2 s_3 - J,
//   f'(J) = -s_1 s_2 s_3 lam (2J - 1) sum_i 1/(q_i s_i) - 1,
// safeguarded by bisection on (1/2, J_max], where c(J_max) = x_3 / (4a) (beyond it
// s_3 is not real).  Then F = B Phi(C), C = B^T B, where Phi is the matrix function
// of phi(x) = s/b = (1 + r(x)) / (2a), r(x) = sqrt(1 - k/x), taken at C's eigenvalues
// x_1 >= x_2 >= x_3 and evaluated as Newton's interpolation polynomial
//   Phi(C) = phi_1 I + phi_12 (C - x_1 I) + phi_123 (C - x_1 I)(C - x_2 I).
// Its divided differences have closed forms free of cancellation (r_i = r(x_i),
// w_i = x_i r_i):
//   phi_12  = k / (2a x_1 x_2 (r_1 + r_2)),
//   phi_123 = -k (r_2 + (x_1 + x_3 - k) / (w_1 + w_3)) / (2a x_1 x_2 x_3 (r_1 + r_2)(r_2 + r_3)),
// so coincident eigenvalues (B near a multiple of a rotation: small strains) need no
// special case, and no eigenvector is formed.  The eigenvalues come from the
// trigonometric solution of C's characteristic cubic.  The cost is a few hundred
// float operations in a few dozen registers, against the assembly and Cholesky
// factorisation of the 9 x 9 Hessian at every step of the general Newton solve.
// Returns false, leaving F as it was, when det B <= 0, when B is badly conditioned
// (x_3 < 4e-3 x_1, where x_3 from C loses its relative accuracy) or when no root is
// found in (1/2, J_max]; the caller then runs the general Newton solve.
__device__ __forceinline__ bool nh3_closed_form(float mu, float lam, float rho, const float* B, float J0, float* F) {
    const float a = mu + rho;
    const float detB = B[0] * (B[4] * B[8] - B[5] * B[7]) + B[1] * (B[5] * B[6] - B[3] * B[8]) +
                       B[2] * (B[3] * B[7] - B[4] * B[6]);
    if (!(detB > 0.f)) return false;
    const float C00 = B[0] * B[0] + B[3] * B[3] + B[6] * B[6];
    const float C11 = B[1] * B[1] + B[4] * B[4] + B[7] * B[7];
    const float C22 = B[2] * B[2] + B[5] * B[5] + B[8] * B[8];
    const float C01 = B[0] * B[1] + B[3] * B[4] + B[6] * B[7];
    const float C02 = B[0] * B[2] + B[3] * B[5] + B[6] * B[8];
    const float C12 = B[1] * B[2] + B[4] * B[5] + B[7] * B[8];
    // eigenvalues of C: m + 2 p cos(theta + 2 pi j / 3), cos(3 theta) = det((C - m I)/p) / 2
    const float m = (C00 + C11 + C22) * (1.f / 3.f);
    const float d0 = C00 - m, d1 = C11 - m, d2 = C22 - m;
    const float p2 = (d0 * d0 + d1 * d1 + d2 * d2 + 2.f * (C01 * C01 + C02 * C02 + C12 * C12)) * (1.f / 6.f);
    float x1 = m, x2 = m, x3 = m;
    if (p2 > 0.f) {
        const float p = sqrtf(p2);
        const float ip = 1.f / p;
        const float e0 = d0 * ip, e1 = d1 * ip, e2 = d2 * ip, e01 = C01 * ip, e02 = C02 * ip, e12 = C12 * ip;
        float h = 0.5f * (e0 * (e1 * e2 - e12 * e12) - e01 * (e01 * e2 - e12 * e02) + e02 * (e01 * e12 - e1 * e02));
        h = fminf(fmaxf(h, -1.f), 1.f);
        float sn, cs;
        __sincosf(acosf(h) * (1.f / 3.f), &sn, &cs);  // |error| < 2^-21 for an angle in [0, pi/3]
        x1 = m + 2.f * p * cs;
        x3 = m - p * (cs + 1.7320508f * sn);
        x2 = 3.f * m - x1 - x3;
    }
    if (!(x3 > 4e-3f * x1)) return false;
    const float b1 = sqrtf(x1), b2 = sqrtf(x2), b3 = sqrtf(x3);
    const float inv2a = 0.5f / a;
    float lo = 0.5f;
    float hi = fminf(0.5f + sqrtf(0.25f + (mu + x3 * (0.25f / a)) / lam), 1e6f);
    float J = (J0 > lo && J0 < hi) ? J0 : 0.5f * (lo + hi);
    bool ok = false;
    for (int it = 0; it < 24; ++it) {
        const float k = 4.f * a * (lam * J * (J - 1.f) - mu);
        // the iterates only steer the root search: fast square roots and quotients
        // (rsqrt, __fdividef) suffice here; the final F below uses IEEE operations
        const float y1 = fmaxf(x1 - k, 1e-30f), y2 = fmaxf(x2 - k, 1e-30f), y3 = fmaxf(x3 - k, 1e-30f);
        const float q1 = y1 * rsqrtf(y1), q2 = y2 * rsqrtf(y2), q3 = y3 * rsqrtf(y3);
        const float s1 = (b1 + q1) * inv2a, s2 = (b2 + q2) * inv2a, s3 = (b3 + q3) * inv2a;
        const float P = s1 * s2 * s3;
        const float fJ = P - J;
        if (fJ == 0.f) {
            ok = true;
            break;
        }
        if (fJ > 0.f)
            lo = J;
        else
            hi = J;
        const float t1 = q1 * s1, t2 = q2 * s2, t3 = q3 * s3;
        const float df = -P * lam * (2.f * J - 1.f) * __fdividef(t2 * t3 + t1 * t3 + t1 * t2, t1 * t2 * t3) - 1.f;
        float Jn = J - __fdividef(fJ, df);
        const bool newton_step = Jn >= lo && Jn <= hi;  // false for NaN
        if (!newton_step) Jn = 0.5f * (lo + hi);
        const float dJ = Jn - J;
        J = Jn;
        if (newton_step && fabsf(dJ) <= 1e-6f * J) {
            ok = true;
            break;
        }
    }
    const float k = 4.f * a * (lam * J * (J - 1.f) - mu);
    if (!ok || !(k < x3)) return false;
    const float q1 = sqrtf(x1 - k), q2 = sqrtf(x2 - k), q3 = sqrtf(x3 - k);
    const float r1 = q1 / b1, r2 = q2 / b2, r3 = q3 / b3;
    const float W = b1 * q1 + b3 * q3;  // w_1 + w_3
    const float D12 = x1 * x2 * (r1 + r2), D23 = x3 * (r2 + r3);
    const float R = 1.f / (D12 * D23 * W);
    const float kh = k * inv2a;
    const float f1 = (1.f + r1) * inv2a;
    const float f123 = -kh * (r2 * W + (x1 + x3 - k)) * R;
    const float g = kh * D23 * W * R + f123 * (x1 - x2);  // phi_12 + phi_123 (x_1 - x_2)
    // Phi(C) = f1 I + g E + phi_123 E^2 with E = C - x_1 I (symmetric)
    const float E00 = C00 - x1, E11 = C11 - x1, E22 = C22 - x1;
    const float M00 = f1 + g * E00 + f123 * (E00 * E00 + C01 * C01 + C02 * C02);
    const float M11 = f1 + g * E11 + f123 * (C01 * C01 + E11 * E11 + C12 * C12);
    const float M22 = f1 + g * E22 + f123 * (C02 * C02 + C12 * C12 + E22 * E22);
    const float M01 = g * C01 + f123 * (E00 * C01 + C01 * E11 + C02 * C12);
    const float M02 = g * C02 + f123 * (E00 * C02 + C01 * C12 + C02 * E22);
    const float M12 = g * C12 + f123 * (C01 * C02 + E11 * C12 + C12 * E22);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float u = B[3 * i], v = B[3 * i + 1], w = B[3 * i + 2];
        F[3 * i + 0] = u * M00 + v * M01 + w * M02;
        F[3 * i + 1] = u * M01 + v * M11 + w * M12;
        F[3 * i + 2] = u * M02 + v * M12 + w * M22;
    }
    return true;
}

// The rare fallback of the closed-form local step: steepest descent with Armijo
// backtracking that keeps J > 0 (Section 2.1's own local method), from the previous
// iterate F.  Few registers beyond F and B, so that the closed-form kernel keeps its
// occupancy.  The step starts at 1/(mu + lam + rho); stops after an accepted step with
// max|dF| <= tol.  Returns the number of steps; conv tells whether the test was met.
template <typename T, int D, typename Law>
__device__ __forceinline__ int steepest_descent(const Law& m, T* F, const T* B, T rho, int cap, T tol, bool& conv) {
    constexpr int NN = D * D;
    conv = false;
    const T t0 = T(1) / (m.mu + m.lam + rho);
    int it = 0;
    for (; it < cap; ++it) {
        T g[NN], aux[Law::NAUX];
        if (!m.grad(F, B, rho, g, aux)) break;
        const T phi0 = m.phi(F, B, rho, aux[NN]);
        T g2 = T(0), gmax = T(0);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            g2 += g[p] * g[p];
            gmax = fmax(gmax, fabs(g[p]));
        }
        T t = t0;
        bool ok = false;
        for (int ls = 0; ls < 30 && !ok; ++ls) {
            T Ft[NN];
#pragma unroll
            for (int p = 0; p < NN; ++p) Ft[p] = F[p] - t * g[p];
            const T Jt = det<T, D>(Ft);
            ok = Jt > T(0) && m.phi(Ft, B, rho, Jt) <= phi0 - T(1e-4) * t * g2;
            if (!ok) t *= T(0.5);
        }
        if (!ok) break;
#pragma unroll
        for (int p = 0; p < NN; ++p) F[p] -= t * g[p];
        if (t * gmax <= tol) {
            conv = true;
            ++it;
            break;
        }
    }
    return it;
}

// W_F(F) - Bm on double-word data for the elastic laws (their grad() in double-word
// arithmetic; F, Bm, g: d*d entries row-major).  False when J <= 0.
template <int D, int MODEL>
__device__ __forceinline__ bool grad_dw(const dw* F, dw mu, dw lam, const dw* Bm, dw* g) {
    constexpr int NN = D * D;
    if constexpr (MODEL == kNeoHooke) {
        dw K[NN], J;
        auto m2 = [&](int a, int b, int c, int d) { return dw_sub(dw_mul(F[a], F[b]), dw_mul(F[c], F[d])); };
        if constexpr (D == 2) {
            K[0] = F[3];
            K[1] = dw_neg(F[2]);
            K[2] = dw_neg(F[1]);
            K[3] = F[0];
            J = m2(0, 3, 1, 2);
        } else {
            K[0] = m2(4, 8, 5, 7);
            K[1] = m2(5, 6, 3, 8);
            K[2] = m2(3, 7, 4, 6);
            K[3] = m2(2, 7, 1, 8);
            K[4] = m2(0, 8, 2, 6);
            K[5] = m2(1, 6, 0, 7);
            K[6] = m2(1, 5, 2, 4);
            K[7] = m2(2, 3, 0, 5);
            K[8] = m2(0, 4, 1, 3);
            J = dw_add(dw_add(dw_mul(F[0], K[0]), dw_mul(F[1], K[1])), dw_mul(F[2], K[2]));
        }
        if (!(J.hi > 0.f)) return false;
        // W_F = mu F + (c / J) K, c = lam J (J - 1) - mu
        const dw cJ = dw_div(dw_sub(dw_mul(dw_mul(lam, J), dw_add_f(J, -1.f)), mu), J);
#pragma unroll
        for (int p = 0; p < NN; ++p) g[p] = dw_sub(dw_add(dw_mul(mu, F[p]), dw_mul(cJ, K[p])), Bm[p]);
        return true;
    } else {
        // W_F = mu (H + H^T) + lam tr(H) I, H = F - I
        dw tr = dw{0.f, 0.f};
#pragma unroll
        for (int i = 0; i < D; ++i) tr = dw_add(tr, dw_add_f(F[i * D + i], -1.f));
        const dw ltr = dw_mul(lam, tr);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j) {
                dw s = dw_add(F[i * D + j], F[j * D + i]);
                if (i == j) s = dw_add_f(s, -2.f);
                dw gij = dw_mul(mu, s);
                if (i == j) gij = dw_add(gij, ltr);
                g[i * D + j] = dw_sub(gij, Bm[i * D + j]);
            }
        return true;
    }
}

// Local step of the double polish, one voxel, in deviation form (elastic laws).
//
// Increment form: with R_k = F_{k+1} - G_k from the previous iteration (float) and
// dG = G_{k+1} - G_k = <F> change + D(u~_{k+1} - u~_k) (float), e = G_{k+1} - F_{k+1}
// = dG - R_k is a float difference of small quantities; r_p sums e^2 and r_d dG^2.
// Multiplier: Lambda_{k+1} = Lambda_k + rho e.  With G = F_{k+1} + e the gradient of
// phi at F_{k+1} is W_F(F) - Bm, Bm = Lambda_{k+1} + rho e: neither G nor
// B = Lambda + rho G is needed.
//
// State: F = Fh + Fl and Lambda = Lh + Ll, pairs of floats whose high parts are held
// fixed while the low parts (the deviations, of the order of the distance the polish
// moves, far below 1) accumulate the updates.  Each pair carries about 48 significant
// bits, like a double-word, without being renormalised after every update.  About Fh
// the gradient is linear to second order:
//   W_F(F) - Bm = Z + W_FF(Fh) Fl - Ll' - rho e + O(|Fl|^2),
//   Z = W_F(Fh) - Lh (formed once in double-word arithmetic and stored as a float),
//   Ll' = Ll + rho e (the new Lambda's low part),
// where every term is small, so float arithmetic gives it to about 1e-7 of its own
// size.  The neglected term is at most |W_FFF| |Fl|^2 / 2; the pair is renormalised
// (two_sum, exact) and Z re-formed whenever max |Fl| exceeds kDevF = 4e-6 (term below
// about 1e-10 |W_FFF| / 100), likewise when max |Ll| exceeds kDevL = 1e-4 (float
// accumulation of Lambda's updates within 1e-11), and on the first step of a polish
// (ctrl->z_valid = 0).  So no double-word arithmetic runs in the common step: the
// earlier form of this step evaluated W_F(F) itself in double-word arithmetic, about
// two thirds of its instructions.
//
// The step is ONE refinement Newton step per iteration, dF = -H_f^{-1} g with the
// float Hessian H_f at Fh, whenever that is a safe full step (no line search, J stays
// positive): F_{k+2} = F_{k+1} + dF and R_{k+1} = F_{k+2} - G_{k+1} = dF - e.  The
// local problem is then solved inexactly, with a gradient left of about
// eps_float cond(H) |g| + c |dF|^2 plus the linearisation term above; in the polish
// |g| and |dF| are of the order of the ADMM residuals, so that error is many orders
// below them and is corrected by the next iteration's step, which starts from this F
// (the inexact local solves of Sections 2.1 and 4.2, r_l << r_d).  A fixed point has
// a local problem stationary to that linearisation error.  Otherwise (a large or
// unsafe step, a failed factorisation: rare, since the polish starts from a converged
// local solve and moves by residual-sized increments) a damped step is taken and the
// following iterations continue from it; a voxel whose Fh is inverted keeps F.
//
// Storage: F as (hi, lo) float arrays in the double F buffers (hi at p V + v, lo at
// (d*d + p) V + v: the same layout as the double-words of the polish's ends), Lambda
// as (Lhi, Llo) updated in place, Z in the idle double Lambda buffer.  The high parts
// change only when renormalised, and then go to both F buffers (the current one is read
// at this voxel by this thread alone): every voxel renormalises on the polish's first
// step, so both buffers hold the same high parts from then on and a common step writes
// only the low parts.  conv tells whether the step was the full refinement step; sp, sd
// get the voxel's squared residual terms.
constexpr float kDevF = 4e-6f;
constexpr float kDevL = 1e-4f;

template <int D, int MODEL, typename I>
__device__ __forceinline__ void polish_voxel_dev(float* __restrict__ Fc, float* __restrict__ Fn,
                                                 float* __restrict__ Lhi, float* __restrict__ Llo,
                                                 float* __restrict__ Zb, float* __restrict__ Rio, const float* dG,
                                                 dw mu, dw lam, float rho, bool fresh, I v, I V,
                                                 float& sp, float& sd, bool& conv) {
    constexpr int NN = D * D;
    constexpr int NP = NN * (NN + 1) / 2;
    using Law = typename LawOf<float, D, MODEL>::type;
    float e[NN], hi[NN], lo[NN], ll[NN], z[NN];
    // neo-Hookean: Z is loaded with the other fields (in the common case it is needed, and
    // a load after the renormalisation test waited for it: 156 -> 146 us per 128^3 launch);
    // the linear law keeps the later load (the early one spills at its register cap)
    constexpr bool kEarlyZ = MODEL == kNeoHooke;
    sp = 0.f;
    sd = 0.f;
    bool ren = fresh;
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        e[p] = dG[p] - Rio[p * V + v];
        sp += e[p] * e[p];
        sd += dG[p] * dG[p];
        hi[p] = Fc[p * V + v];
        lo[p] = Fc[(NN + p) * V + v];
        ll[p] = Llo[p * V + v];
        if constexpr (kEarlyZ) z[p] = Zb[p * V + v];
        ren |= fabsf(lo[p]) > kDevF || fabsf(ll[p]) > kDevL;
    }
    if (ren) {  // rare: renormalise both pairs, Z from the new high parts
        dw F[NN], Bm[NN], g[NN];
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            const dw f = two_sum(hi[p], lo[p]);
            const dw l = two_sum(Lhi[p * V + v], ll[p]);
            hi[p] = f.hi;
            lo[p] = f.lo;
            ll[p] = l.lo;
            Lhi[p * V + v] = l.hi;
            Fc[p * V + v] = f.hi;
            Fn[p * V + v] = f.hi;
            F[p] = dw{f.hi, 0.f};
            Bm[p] = dw{l.hi, 0.f};
        }
        const bool ok = grad_dw<D, MODEL>(F, mu, lam, Bm, g);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            z[p] = ok ? g[p].hi : 0.f;
            Zb[p * V + v] = z[p];
        }
    } else if constexpr (!kEarlyZ) {
#pragma unroll
        for (int p = 0; p < NN; ++p) z[p] = Zb[p * V + v];
    }
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        ll[p] += rho * e[p];  // Lambda_{k+1} - Lh
        Llo[p * V + v] = ll[p];
    }
    const Law m{mu.hi, lam.hi};
    float aux[Law::NAUX];
    if constexpr (MODEL == kNeoHooke) aux[NN] = det_cof<float, D>(hi, aux);
    else aux[0] = 1.f;
    conv = false;
    if (MODEL != kNeoHooke || aux[NN] > 0.f) {
        float Hf[NP], gf[NN], df[NN];
        m.hess(aux, rho, Hf);
        // g = Z + (H_f - rho I) Fl - Ll' - rho e, H_f packed lower
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            float w = -rho * lo[p];
#pragma unroll
            for (int q = 0; q < NN; ++q) w += Hf[p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p] * lo[q];
            gf[p] = (z[p] + w) - (ll[p] + rho * e[p]);
        }
        const bool ok = chol_solve<float, NN>(Hf, gf, df);
        float slope = 0.f, size = 0.f;
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            slope += gf[p] * df[p];
            size = fmaxf(size, fabsf(df[p]));
        }
        float t = 1.f;
        if (ok && slope < 0.f && size <= NewtonConst<float>::big && m.small_step_safe(aux, size)) {
            conv = true;  // the one refinement step
        } else {
            // Rare (a large or unsafe step, a failed factorisation): a damped step
            // instead of a full local solve -- the Newton direction, or steepest descent
            // where that does not descend, shortened to the trust size and halved until J
            // stays positive; the next iteration continues from it.
            if (!(ok && slope < 0.f)) {
                const float sc = 1.f / (mu.hi + rho);
                size = 0.f;
#pragma unroll
                for (int p = 0; p < NN; ++p) {
                    df[p] = -gf[p] * sc;
                    size = fmaxf(size, fabsf(df[p]));
                }
            }
            t = size > NewtonConst<float>::big ? NewtonConst<float>::big / size : 1.f;
            int h = 0;
            for (; h < 30; ++h) {
                float Ft[NN];
#pragma unroll
                for (int p = 0; p < NN; ++p) Ft[p] = hi[p] + (lo[p] + t * df[p]);
                if (det<float, D>(Ft) > 0.f) break;
                t *= 0.5f;
            }
            if (h == 30 || !(size < 1e30f)) t = 0.f;
        }
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            lo[p] += t * df[p];
            e[p] = t * df[p] - e[p];
        }
    } else {
#pragma unroll
        for (int p = 0; p < NN; ++p) e[p] = -e[p];  // inverted state: F stays, R_{k+1} = -e
    }
#pragma unroll
    for (int p = 0; p < NN; ++p) {
        Fn[(NN + p) * V + v] = lo[p];
        Rio[p * V + v] = e[p];
    }
}

// ------------------------------------------------------------------ liquid crystal elastomer
// Section 5.1 with the readings of the oracle: compressible network with the
// positive-definite step-length tensor l = r^{-1/3}(I + (r-1) n n), non-ideality,
// Frank gradient from the previous iterate.  With m = F^T n and
// M = c1 I - c2 n0 n0 (c1 = mu(alpha - r^{1/3}(1 - 1/r)), c2 = mu alpha):
//   W = a/2 |F|^2 + 1/2 m.M m - mu ln J + lam/2 (J-1)^2 + const,   a = mu r^{1/3}.
// Local objective: phi(F, n) = W - f.n - Lambda:F + rho/2 |F - G|^2 on |n| = 1,
// f = 2 kappa_F / h^2 * (sum of the neighbours' directors of the previous iterate).
// The incompressible network (inc) drops the volumetric terms (muv = lam = 0): its
// constraint det F = 1 is the local step's (newton_lce_inc).
template <typename T>
struct Lce {
    T mu, lam, a, c1, c2;
    T muv;  // coefficient of -ln J: mu, or 0 for the incompressible network
    T n0[3];
    __device__ __forceinline__ void Mv(const T* v, T* o) const {
        const T d = n0[0] * v[0] + n0[1] * v[1] + n0[2] * v[2];
        for (int i = 0; i < 3; ++i) o[i] = c1 * v[i] - c2 * d * n0[i];
    }
    __device__ __forceinline__ T phi(const T* F, const T* n, const T* B, const T* f, T rho, T J) const {
        T ff = 0, bf = 0, mm[3], Mm[3];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            ff += F[p] * F[p];
            bf += B[p] * F[p];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) mm[j] = n[0] * F[j] + n[1] * F[3 + j] + n[2] * F[6 + j];
        Mv(mm, Mm);
        const T q = mm[0] * Mm[0] + mm[1] * Mm[1] + mm[2] * Mm[2];
        return T(0.5) * (a + rho) * ff + T(0.5) * q - muv * log_t(J) + T(0.5) * lam * (J - T(1)) * (J - T(1)) -
               (f[0] * n[0] + f[1] * n[1] + f[2] * n[2]) - bf;
    }
    // W_F = a F + n (x) M m + (lam J (J-1) - muv) F^{-T}
    __device__ __forceinline__ void stress(const T* F, const T* n, T* P) const {
        T K[9], mm[3], Mm[3];
        const T J = det_cof<T, 3>(F, K);
        const T c = (lam * J * (J - T(1)) - muv) / J;
#pragma unroll
        for (int j = 0; j < 3; ++j) mm[j] = n[0] * F[j] + n[1] * F[3 + j] + n[2] * F[6 + j];
        Mv(mm, Mm);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) P[k * 3 + l] = a * F[k * 3 + l] + n[k] * Mm[l] + c * K[k * 3 + l];
    }
};

template <typename T, bool INC = false>
__device__ __forceinline__ Lce<T> load_lce(const uint8_t* phase, const T* mat, int nparam, long long v,
                                          const T* __restrict__ n0, long long V) {
    const int ph = phase[v];
    const T* q = mat + ph * nparam;
    Lce<T> m;
    m.mu = __ldg(q + 0);
    m.lam = INC ? T(0) : __ldg(q + 1);
    m.muv = INC ? T(0) : m.mu;
    m.a = __ldg(q + 5);
    m.c1 = __ldg(q + 6);
    m.c2 = __ldg(q + 7);
    m.n0[0] = n0[v];
    m.n0[1] = n0[V + v];
    m.n0[2] = n0[2 * V + v];
    return m;
}

// Orthonormal (ta, tb) spanning the tangent plane at the unit vector n.
template <typename T>
__device__ __forceinline__ void tangent_basis(const T* n, T* ta, T* tb) {
    const T ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
    T e[3] = {T(0), T(0), T(0)};
    if (ax <= ay && ax <= az) e[0] = T(1);
    else if (ay <= az) e[1] = T(1);
    else e[2] = T(1);
    const T d = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
    T nrm = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ta[i] = e[i] - d * n[i];
        nrm += ta[i] * ta[i];
    }
    const T inv = T(1) / sqrt(nrm);
#pragma unroll
    for (int i = 0; i < 3; ++i) ta[i] *= inv;
    tb[0] = n[1] * ta[2] - n[2] * ta[1];
    tb[1] = n[2] * ta[0] - n[0] * ta[2];
    tb[2] = n[0] * ta[1] - n[1] * ta[0];
}

template <typename T>
__device__ __forceinline__ void retract(const T* n, const T* ta, const T* tb, T t1, T t2, T* out) {
    T nrm = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        out[i] = n[i] + t1 * ta[i] + t2 * tb[i];
        nrm += out[i] * out[i];
    }
    const T inv = T(1) / sqrt(nrm);
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] *= inv;
}

// Hessian of phi in (F, t1, t2) at (F, n), packed lower triangle, in float:
// F-F block diag I + n_k n_r M_ls + bv A_kl A_rs - cv A_ks A_rl (A = F^{-T}), F-t rows
// e_r (M m)_s + n_r (M F^T e)_s, t-t block (F^T e).M (F^T e') + shift I.
template <typename T>
__device__ __forceinline__ void lce_hessian(const Lce<T>& m, const T* F, const T* n, const T* ta, const T* tb,
                                            const T* A, const T* Mm, float bv, float cv, float diag, float shift,
                                            float* H) {
    float Af[9], nf[3], n0f[3], Mmf[3], Ftaf[3], Ftbf[3], MFta[3], MFtb[3];
    const float c1 = (float)m.c1, c2 = (float)m.c2;
#pragma unroll
    for (int p = 0; p < 9; ++p) Af[p] = (float)A[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        nf[i] = (float)n[i];
        n0f[i] = (float)m.n0[i];
        Mmf[i] = (float)Mm[i];
    }
    // F^T ta, F^T tb and M applied to them
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Ftaf[j] = (float)(F[j] * ta[0] + F[3 + j] * ta[1] + F[6 + j] * ta[2]);
        Ftbf[j] = (float)(F[j] * tb[0] + F[3 + j] * tb[1] + F[6 + j] * tb[2]);
    }
    {
        const float da = n0f[0] * Ftaf[0] + n0f[1] * Ftaf[1] + n0f[2] * Ftaf[2];
        const float db = n0f[0] * Ftbf[0] + n0f[1] * Ftbf[1] + n0f[2] * Ftbf[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            MFta[i] = c1 * Ftaf[i] - c2 * da * n0f[i];
            MFtb[i] = c1 * Ftbf[i] - c2 * db * n0f[i];
        }
    }
    // F-F block
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int k = p / 3, l = p % 3;
#pragma unroll
        for (int q = 0; q <= p; ++q) {
            const int r = q / 3, s2 = q % 3;
            const float Mls = (l == s2 ? c1 : 0.f) - c2 * n0f[l] * n0f[s2];
            float h = nf[k] * nf[r] * Mls + bv * Af[p] * Af[q] - cv * Af[k * 3 + s2] * Af[r * 3 + l];
            if (p == q) h += diag;
            H[p * (p + 1) / 2 + q] = h;
        }
    }
    // director rows: d2/dF_rs dt_beta = e_r (M m)_s + n_r (M F^T e)_s
    const float taf[3] = {(float)ta[0], (float)ta[1], (float)ta[2]};
    const float tbf[3] = {(float)tb[0], (float)tb[1], (float)tb[2]};
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int r = q / 3, s2 = q % 3;
        H[9 * 10 / 2 + q] = taf[r] * Mmf[s2] + nf[r] * MFta[s2];
        H[10 * 11 / 2 + q] = tbf[r] * Mmf[s2] + nf[r] * MFtb[s2];
    }
    H[9 * 10 / 2 + 9] = Ftaf[0] * MFta[0] + Ftaf[1] * MFta[1] + Ftaf[2] * MFta[2] + shift;
    H[10 * 11 / 2 + 9] = Ftbf[0] * MFta[0] + Ftbf[1] * MFta[1] + Ftbf[2] * MFta[2];
    H[10 * 11 / 2 + 10] = Ftbf[0] * MFtb[0] + Ftbf[1] * MFtb[1] + Ftbf[2] * MFtb[2] + shift;
}

// Newton on (F, t1, t2) with n <- normalise(n + t1 ta + t2 tb) (tangent plane at the
// current n): gradient and objective in T, Hessian (11x11) assembled and factored
// in float; the director block gets the curvature term -(n . phi_n) I and a shift
// 1e-6 mu I (a Levenberg term that keeps the step defined where W does not depend
// on n; the converged point is unchanged).  Same line search and stopping rule as
// newton().
template <typename T>
__device__ __forceinline__ int newton_lce(const Lce<T>& m, T* F, T* n, const T* B, const T* f, T rho, int cap, T tol,
                                          bool& conv, T gtol = T(0), T* gnorm2 = nullptr) {
    constexpr int NU = 11;
    constexpr int NP = NU * (NU + 1) / 2;
    conv = false;
    int it = 0;
    bool small = false;  // as in newton()
    while (it < cap || small) {
        T A[9], mm[3], Mm[3], g[NU], ta[3], tb[3];
        const T J = det_cof<T, 3>(F, A);
        if (!(J > T(0))) break;
        const T iJ = T(1) / J;
#pragma unroll
        for (int p = 0; p < 9; ++p) A[p] *= iJ;
#pragma unroll
        for (int j = 0; j < 3; ++j) mm[j] = n[0] * F[j] + n[1] * F[3 + j] + n[2] * F[6 + j];
        m.Mv(mm, Mm);
        const T c = m.lam * J * (J - T(1)) - m.muv;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l)
                g[k * 3 + l] = (m.a + rho) * F[k * 3 + l] + n[k] * Mm[l] + c * A[k * 3 + l] - B[k * 3 + l];
        T gn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gn[k] = F[k * 3 + 0] * Mm[0] + F[k * 3 + 1] * Mm[1] + F[k * 3 + 2] * Mm[2] - f[k];
        tangent_basis(n, ta, tb);
        g[9] = ta[0] * gn[0] + ta[1] * gn[1] + ta[2] * gn[2];
        g[10] = tb[0] * gn[0] + tb[1] * gn[1] + tb[2] * gn[2];
        const T ngn = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];
        if (gtol > T(0)) {
            T s2 = T(0);
#pragma unroll
            for (int p = 0; p < NU; ++p) s2 += g[p] * g[p];
            *gnorm2 = s2;
            if (small || s2 <= gtol * gtol) {
                conv = true;
                break;
            }
        }

        float d[NU], gf[NU];
#pragma unroll
        for (int p = 0; p < NU; ++p) gf[p] = (float)g[p];
        {
            float H[NP];
            const float Jf = (float)J;
            lce_hessian<T>(m, F, n, ta, tb, A, Mm, (float)m.lam * (2.f * Jf - 1.f) * Jf, (float)c, (float)(m.a + rho),
                           1e-6f * (float)m.mu - (float)ngn, H);
            if (!chol_solve<float, NU>(H, gf, d)) {
                const float sc = 1.f / (float)(m.mu + rho);
#pragma unroll
                for (int p = 0; p < NU; ++p) d[p] = -gf[p] * sc;
            }
        }
        float slope = 0.f, size = 0.f;
#pragma unroll
        for (int p = 0; p < NU; ++p) {
            slope += gf[p] * d[p];
            size = fmaxf(size, fabsf(d[p]));
        }
        if (!(slope < 0.f)) {
            const float sc = 1.f / (float)(m.mu + rho);
            slope = 0.f;
            size = 0.f;
#pragma unroll
            for (int p = 0; p < NU; ++p) {
                d[p] = -gf[p] * sc;
                slope += gf[p] * d[p];
                size = fmaxf(size, fabsf(d[p]));
            }
        }
        if (!(size < 1e30f)) break;
        T t = T(1);
        T Ft[9], nt[3];
        {
            const T phi0 = (size > (float)NewtonConst<T>::big) ? m.phi(F, n, B, f, rho, J) : T(0);
            int ls = 0;
            for (; ls < 40; ++ls) {
#pragma unroll
                for (int p = 0; p < 9; ++p) Ft[p] = F[p] + t * (T)d[p];
                const T Jt = det<T, 3>(Ft);
                if (Jt > T(0)) {
                    if (!(size > (float)NewtonConst<T>::big)) break;
                    retract(n, ta, tb, t * (T)d[9], t * (T)d[10], nt);
                    if (m.phi(Ft, nt, B, f, rho, Jt) <= phi0 + T(1e-4) * t * (T)slope) break;
                }
                t *= T(0.5);
            }
            if (ls == 40) t = T(0);
        }
#pragma unroll
        for (int p = 0; p < 9; ++p) F[p] += t * (T)d[p];
        retract(n, ta, tb, t * (T)d[9], t * (T)d[10], nt);
#pragma unroll
        for (int i = 0; i < 3; ++i) n[i] = nt[i];
        ++it;
        if (t == T(1) && size <= (float)tol) {
            if (gtol > T(0)) {
                small = true;
                continue;
            }
            conv = true;
            break;
        }
        if (t == T(0)) break;
    }
    return it;
}

// The incompressible network (Section 5.1, det F = 1 by a multiplier p of the local
// step): Newton on the stationarity of phi - p (det F - 1) in (F, t1, t2, p).  Each step
// solves the KKT system [[K, -c], [-c^T, 0]] (dx, dp) = (-g, J - 1), c = (cof F, 0, 0),
// K = phi's Hessian in (F, t) with -p d2(det) on the F block (float), by its Schur
// complement on p: with y = K^-1 g and z = K^-1 c, dp = (c.y - (J - 1)) / (c.z) and
// dx = dp z - y.  Where K is not positive definite (its Cholesky factorisation fails:
// the director near a maximum) (mu + rho_pen) I is added.  p starts from the
// least-squares fit of cof F to phi's F-gradient; steps longer than kIncBig are scaled
// to it and halved while det F <= 0; no merit line search.  Stops after a full step
// of size <= tol.  rho: F-penalty including the dissipation weight; rho_pen: ADMM rho.
constexpr float kIncBig = 0.25f;  // longest step (max norm over F and t) of newton_lce_inc

template <typename T>
__device__ __forceinline__ int newton_lce_inc(const Lce<T>& m, T* F, T* n, const T* B, const T* f, T rho, T rho_pen,
                                              int cap, T tol, bool& conv) {
    constexpr int NU = 11;
    constexpr int NP = NU * (NU + 1) / 2;
    conv = false;
    T pm = T(0);
    int it = 0;
    while (it < cap) {
        T C[9], A[9], mm[3], Mm[3], g[NU], ta[3], tb[3];
        const T J = det_cof<T, 3>(F, C);
        if (!(J > T(0))) break;
        const T iJ = T(1) / J;
#pragma unroll
        for (int q = 0; q < 9; ++q) A[q] = C[q] * iJ;
#pragma unroll
        for (int j = 0; j < 3; ++j) mm[j] = n[0] * F[j] + n[1] * F[3 + j] + n[2] * F[6 + j];
        m.Mv(mm, Mm);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = 0; l < 3; ++l) g[k * 3 + l] = (m.a + rho) * F[k * 3 + l] + n[k] * Mm[l] - B[k * 3 + l];
        if (it == 0) {
            T cc = T(0), cg = T(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                cc += C[q] * C[q];
                cg += C[q] * g[q];
            }
            pm = cg / cc;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] -= pm * C[q];
        T gn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gn[k] = F[k * 3 + 0] * Mm[0] + F[k * 3 + 1] * Mm[1] + F[k * 3 + 2] * Mm[2] - f[k];
        tangent_basis(n, ta, tb);
        g[9] = ta[0] * gn[0] + ta[1] * gn[1] + ta[2] * gn[2];
        g[10] = tb[0] * gn[0] + tb[1] * gn[1] + tb[2] * gn[2];
        const T ngn = n[0] * gn[0] + n[1] * gn[1] + n[2] * gn[2];

        float d[NU], dp;
        {
            float H[NP], inv[NU], gf[NU], cf[NU], y[NU], z[NU];
#pragma unroll
            for (int q = 0; q < NU; ++q) {
                gf[q] = (float)g[q];
                cf[q] = q < 9 ? (float)C[q] : 0.f;
            }
            const float pJ = (float)(pm * J), diag = (float)(m.a + rho);
            const float shift = 1e-6f * (float)m.mu - (float)ngn;
            lce_hessian<T>(m, F, n, ta, tb, A, Mm, -pJ, -pJ, diag, shift, H);
            if (!chol_factor<float, NU>(H, inv)) {
                const float sh = (float)(m.mu + rho_pen);
                lce_hessian<T>(m, F, n, ta, tb, A, Mm, -pJ, -pJ, diag + sh, shift + sh, H);
                if (!chol_factor<float, NU>(H, inv)) break;
            }
            chol_subst<float, NU>(H, inv, gf, y);  // -K^-1 g
            chol_subst<float, NU>(H, inv, cf, z);  // -K^-1 c
            float cy = 0.f, cz = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                cy += cf[q] * y[q];
                cz += cf[q] * z[q];
            }
            dp = (cy + (float)(J - T(1))) / cz;
#pragma unroll
            for (int q = 0; q < NU; ++q) d[q] = y[q] - dp * z[q];
        }
        float size = 0.f;
#pragma unroll
        for (int q = 0; q < NU; ++q) size = fmaxf(size, fabsf(d[q]));
        if (!(size < 1e30f) || !(fabsf(dp) < 1e30f)) break;
        T t = size > kIncBig ? T(kIncBig) / (T)size : T(1);
        T Ft[9];
        int h = 0;
        for (; h < 40; ++h) {
#pragma unroll
            for (int q = 0; q < 9; ++q) Ft[q] = F[q] + t * (T)d[q];
            if (det<T, 3>(Ft) > T(0)) break;
            t *= T(0.5);
        }
        if (h == 40) break;
        T nt[3];
        retract(n, ta, tb, t * (T)d[9], t * (T)d[10], nt);
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = Ft[q];
#pragma unroll
        for (int i = 0; i < 3; ++i) n[i] = nt[i];
        pm += t * (T)dp;
        ++it;
        if (t == T(1) && size <= (float)tol) {
            conv = true;
            break;
        }
    }
    return it;
}

// ------------------------------------------------------------------ grid helpers

// Periodic neighbour indices of voxel v (x fastest).  32-bit arithmetic: one
// RVE has at most 512^3 < 2^31 voxels, and 64-bit division would run as a long
// software sequence on every voxel.
template <int D>
struct Nbr {
    int xp, xm, yp, ym, zp, zm;
};

template <int D>
__device__ __forceinline__ Nbr<D> neighbours(int v, const FastDiv& dn) {
    Nbr<D> o;
    const int n = (int)dn.d;
    const unsigned un = dn.d;
    const unsigned r = fdiv((unsigned)v, dn);
    const int x = v - (int)(r * un);
    o.xp = v + (x + 1 == n ? 1 - n : 1);
    o.xm = v + (x == 0 ? n - 1 : -1);
    if constexpr (D == 3) {
        const unsigned zq = fdiv(r, dn);
        const int y = (int)(r - zq * un);
        const int z = (int)zq;
        o.yp = v + (y + 1 == n ? (1 - n) * n : n);
        o.ym = v + (y == 0 ? (n - 1) * n : -n);
        const int s2 = n * n;
        o.zp = v + (z + 1 == n ? (1 - n) * s2 : s2);
        o.zm = v + (z == 0 ? (n - 1) * s2 : -s2);
    } else {
        const int y = (int)r;
        o.yp = v + (y + 1 == n ? (1 - n) * n : n);
        o.ym = v + (y == 0 ? (n - 1) * n : -n);
        o.zp = o.zm = v;
    }
    return o;
}

// G_ij = Fbar_ij + (u_i(x + h e_j) - u_i(x - h e_j)) / (2h), h = 1/n.
template <typename T, int D>
__device__ __forceinline__ void grad_u(const T* __restrict__ U, long long V, const Nbr<D>& nb, const T* Fb,
                                       T half_n, T* G) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const T* u = U + i * V;
        G[i * D + 0] = Fb[i * D + 0] + (__ldg(u + nb.xp) - __ldg(u + nb.xm)) * half_n;
        G[i * D + 1] = Fb[i * D + 1] + (__ldg(u + nb.yp) - __ldg(u + nb.ym)) * half_n;
        if constexpr (D == 3) G[i * D + 2] = Fb[i * D + 2] + (__ldg(u + nb.zp) - __ldg(u + nb.zm)) * half_n;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------ kernels

// Director fields of the LCE (null for the other laws): ping-pong N0/N1 by the
// same parity as F, and the reference directors n0 (read only).
template <typename T>
struct Dirs {
    T* N0;
    T* N1;
    const T* ref;
    const T* Fp;  // previous time step (dissipation): F and n
    const T* np;
};

template <typename T>
struct Set;
template <>
struct Set<double> {
    __host__ __device__ static double* F(const Launch& L, int i) { return L.F64[i]; }
    __host__ __device__ static double* Lm(const Launch& L) { return L.L64; }
    __host__ __device__ static double* U(const Launch& L, int i) { return L.U64[i]; }
    __host__ __device__ static Dirs<double> dirs(const Launch& L) {
        return Dirs<double>{L.N64[0], L.N64[1], L.n0_64, L.Fp64, L.np64};
    }
    __host__ __device__ static const double* mat(const Launch& L) { return L.mat; }
    __host__ __device__ static double half_n(const Launch& L) { return L.half_n64; }
    __host__ __device__ static double two_nsq(const Launch& L) { return L.two_nsq64; }
};
template <>
struct Set<float> {
    __host__ __device__ static float* F(const Launch& L, int i) { return L.F32[i]; }
    __host__ __device__ static float* Lm(const Launch& L) { return L.L32; }
    __host__ __device__ static float* U(const Launch& L, int i) { return L.U32[i]; }
    __host__ __device__ static Dirs<float> dirs(const Launch& L) {
        return Dirs<float>{L.N32[0], L.N32[1], L.n0_32, L.Fp32, L.np32};
    }
    __host__ __device__ static const float* mat(const Launch& L) { return L.mat32; }
    __host__ __device__ static float half_n(const Launch& L) { return L.half_n32; }
    __host__ __device__ static float two_nsq(const Launch& L) { return L.two_nsq32; }
};

// Fresh state: F_k = Fbar, u~_k = 0, Lambda = W_F(Fbar; x) (or 0).
template <typename T, int D, int MODEL>
__global__ void __launch_bounds__(kLocalThreads)
k_init(const Ctrl* __restrict__ ctrl, T* F0, T* F1, T* Lam, T* U0, T* U1, const uint8_t* __restrict__ phase,
       const T* __restrict__ mat, int nparam, long long V, int lambda_zero, Dirs<T> dir) {
    const int par = (int)(ctrl->k & 1);
    T* F = par ? F1 : F0;
    T* U = par ? U1 : U0;
    T Fb[D * D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) Fb[i * D + j] = (T)ctrl->Fbar[i * 3 + j];
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        T P[D * D];
        if constexpr (is_lce(MODEL)) {
            T* Nk = par ? dir.N1 : dir.N0;
            T nv[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                nv[i] = dir.ref[i * V + v];
                Nk[i * V + v] = nv[i];
            }
            if (lambda_zero) {
#pragma unroll
                for (int p = 0; p < 9; ++p) P[p] = T(0);
            } else {
                load_lce<T, MODEL == kLceInc>(phase, mat, nparam, v, dir.ref, V).stress(Fb, nv, P);
            }
        } else if (lambda_zero) {
#pragma unroll
            for (int p = 0; p < D * D; ++p) P[p] = T(0);
        } else {
            using Law = typename LawOf<T, D, MODEL>::type;
            const Law m = load_law<Law, T>(phase, mat, nparam, v);
            m.stress(Fb, P);
        }
#pragma unroll
        for (int p = 0; p < D * D; ++p) {
            F[p * V + v] = Fb[p];
            Lam[p * V + v] = P[p];
        }
#pragma unroll
        for (int i = 0; i < D; ++i) U[i * V + v] = T(0);
    }
}

// End of one tile of the fused pass (not the local-step-only pass): block sums of the
// thread partials r_p^2, r_d^2, r_l^2 (warp sums in the threads' accumulator type, float
// in the float kernels, whose FP64 pipe is 1/64 of the FP32 rate; sums across warps and
// tiles in double), the largest Newton count and the failures go to the tile's slot of
// the partial buffer; the last tile of the RVE to
// finish (atomic counter) sums all slots in a fixed order, so the result does not
// depend on block scheduling, and runs the control step: residuals of iteration k,
// stop flag, precision switch, adaptive rho.  INC: the increment form of the polish.
// spec: the voxel sums of |G_{k+1} - G_k|^2 come from the z pass's tile sums zpart (nz of
// them; see Launch::Sprev) instead of the threads' r_d partials.
template <int D, bool INC, typename Acc>
__device__ __forceinline__ void finish_pass(Ctrl* __restrict__ ctrl, double* __restrict__ hist,
                                            double* __restrict__ partials, int bid, int nblk, long long V,
                                            long long k, Acc rp2a, Acc rd2a, Acc rl2a, int nmax, int nfail,
                                            bool frac_on, const int* s_hist, bool spec = false,
                                            const double* zpart = nullptr, int nz = 0) {
    __shared__ double s_sum[kLocalThreads / 32][3];
    __shared__ int s_int[kLocalThreads / 32][2];
    __shared__ int s_last;

    // block partials: r_p^2, r_d^2 sums (double), Newton max / failures
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double rp2 = (double)warp_sum(rp2a);
    const double rd2 = (double)warp_sum(rd2a);
    const double rl2 = (double)warp_sum(rl2a);
    nmax = warp_max(nmax);
    for (int o = 16; o > 0; o >>= 1) nfail += __shfl_down_sync(0xffffffffu, nfail, o);
    if (lane == 0) {
        s_sum[warp][0] = rp2;
        s_sum[warp][1] = rd2;
        s_sum[warp][2] = rl2;
        s_int[warp][0] = nmax;
        s_int[warp][1] = nfail;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, cl = 0;
        int mx = 0, nf = 0;
        for (int w = 0; w < kLocalThreads / 32; ++w) {
            a += s_sum[w][0];
            b += s_sum[w][1];
            cl += s_sum[w][2];
            mx = max(mx, s_int[w][0]);
            nf += s_int[w][1];
        }
        double* pp = partials + (size_t)bid * kPartialStride;
        pp[0] = a;
        pp[1] = b;
        pp[2] = (double)mx;
        pp[3] = (double)nf;
        pp[4] = cl;
        if (frac_on)
            for (int b = 0; b < kNewtonBins; ++b)
                if (s_hist[b]) atomicAdd(&ctrl->newton_hist[b], (unsigned)s_hist[b]);
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->counter, 1u);
        s_last = (prev == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last block: fixed-order sum over all block partials
    double a = 0, b = 0, cl = 0;
    int mx = 0;
    double nf = 0;
    for (int i = threadIdx.x; i < (int)nblk; i += blockDim.x) {
        const double* pp = partials + (size_t)i * kPartialStride;
        a += __ldcg(pp + 0);
        b += __ldcg(pp + 1);
        mx = max(mx, (int)__ldcg(pp + 2));
        nf += __ldcg(pp + 3);
        cl += __ldcg(pp + 4);
    }
    if (spec) {
        // Parseval: sum_x |D w|^2 = (1/V) sum_m |k_m|^2 |w^(m)|^2 for the true DFT w^, and the
        // z pass holds u^ scaled by 2/V, so the voxel sum is V/4 times its tile sums
        double zb = 0.0;
        for (int i = threadIdx.x; i < nz; i += blockDim.x) zb += __ldcg(zpart + i);
        b += 0.25 * (double)V * zb;
    }
    a = warp_sum(a);
    b = warp_sum(b);
    cl = warp_sum(cl);
    nf = warp_sum(nf);
    mx = warp_max(mx);
    if (lane == 0) {
        s_sum[warp][0] = a;
        s_sum[warp][1] = b;
        s_sum[warp][2] = cl;
        s_int[warp][0] = mx;
        s_int[warp][1] = (int)nf;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    a = 0;
    b = 0;
    cl = 0;
    mx = 0;
    long long nft = 0;
    for (int w = 0; w < kLocalThreads / 32; ++w) {
        a += s_sum[w][0];
        b += s_sum[w][1];
        cl += s_sum[w][2];
        mx = max(mx, s_int[w][0]);
        nft += s_int[w][1];
    }
    Ctrl* c = ctrl;
    const double rhod = c->rho;
    if (!INC) {
        double dm = 0.0;  // |<F>_{k+1} - <F>_k|^2 (mixed control)
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                const double x = c->Fbar[i * 3 + j] - c->Fbar_prev[i * 3 + j];
                dm += x * x;
            }
        b += dm * (double)V;
    }
    const double r_p = sqrt(a / (double)V);
    const double r_d = rhod / c->mu_ref * sqrt(b / (double)V);
    const long long idx = k - c->k_start;
    const double r_l = sqrt(cl / (double)V) / c->mu_ref;
    if (idx >= 0 && idx < c->hist_cap) {
        hist[kHistStride * idx + 0] = r_p;
        hist[kHistStride * idx + 1] = r_d;
        hist[kHistStride * idx + 2] = rhod;
        hist[kHistStride * idx + 3] = r_l;
    }
    c->r_p = r_p;
    c->rd_local = c->r_d;
    c->r_d = r_d;
    c->r_l = r_l;
    c->k = k + 1;
    c->newton_max = mx;
    c->newton_fail = (unsigned long long)nft;
    if (frac_on) {
        // the smallest even count by which a fraction p of the voxels converged; if
        // fewer converged within the cap, raise the cap by 2 (up to the configured one)
        const double need = c->local_fraction * (double)V;
        int cap_next = min(c->newton_cap + 2, c->newton_cap_max);
        double cum = 0.0;
        bool found = false;
        for (int bin = 0; bin < kNewtonBins; ++bin) {
            cum += (double)__ldcg(&c->newton_hist[bin]);
            if (!found && cum >= need) {
                cap_next = min(2 * (bin + 1), c->newton_cap_max);
                found = true;
            }
            c->newton_hist[bin] = 0u;
        }
        c->newton_cap = cap_next;
    }
    int done = kRunning;
    if (!(isfinite(r_p) && isfinite(r_d))) {
        done = kNumerical;
    } else if (r_p <= c->tol && r_d <= c->tol) {
        done = kConverged;
    } else if (k + 1 >= c->k_cap) {
        done = kCapped;
    } else if (c->phase_fp32) {
        const double mres = fmax(r_p, r_d);
        if (mres <= c->switch_tol) {
            done = kSwitch;
        } else if (mres < 0.9 * c->best) {
            c->best = mres;
            c->stall = 0;
        } else if (++c->stall >= 10) {
            done = kSwitch;
        }
    }
    c->rho_changed = 0;
    c->div_given = 0;  // the switch's divergence has been transformed by now
    c->spec_have = c->spec_next;  // the z pass of this iteration stored u^_{k+1}
    c->spec_next = 0;
    c->spec_sum = 0;
    if (INC) c->z_valid = 1;  // the polish's first step has formed Z at every voxel
    if (done == kRunning && c->adaptive) {  // eq. rho-update (He, Yang & Wang)
        double nr = rhod;
        if (r_d > 0.0 && r_p / r_d > c->rho_tau)
            nr = c->rho_kappa * rhod;
        else if (r_p > 0.0 && r_d / r_p > c->rho_tau)
            nr = fmax(rhod / c->rho_kappa, c->rho_min);
        if (nr != rhod) {
            c->rho = nr;
            c->inv_rho = 1.0 / nr;
            c->rho_changed = 1;
        }
    }
    c->done = done;
    c->counter = 0u;
}

// The fused per-iteration kernel.  With FIRST = false, at iteration index k
// (k iterations done): reads u~_{k+1}, u~_k, F_{k+1}, Lambda_k; writes
// Lambda_{k+1} (Step 3), accumulates r_p, r_d of iteration k (Step 4) and runs
// Step 1 of iteration k+1 into F_{k+2}; the last block finishes the residuals,
// advances k and sets the stop flag.  With FIRST = true only Step 1 runs
// (F_{k+1} from F_k, Lambda_k, u~_k): at the start of a solve, after a precision
// switch, and (only_if_rho_changed) to redo the speculative step when the
// adaptive rule changed rho.
//
// WRITE_R (double polish of RVE_MIXED): also store R = F_{k+2} - G_{k+1} in
// float.  With rho fixed, Q_{k+2} - Q_{k+1} = R for Q = F - Lambda/rho, so the
// next projection only has to transform this small increment (see rve_fft.cu).
//
// DU (same polish, after its first iteration): the float increment
// u~_{k+1} - u~_k written by the increment projection is read instead of u~_k,
// and G_{k+1} - G_k = D(u~_{k+1} - u~_k) for r_d is formed in float.  For the
// elastic laws this iteration runs in increment form on pairs of floats (INC,
// polish_voxel_dev): F and Lambda are float pairs, and at ctrl->k = k the state
// F_{k+1} sits in F buffer k & 1 (one parity off the double convention) so that
// the conversions at the polish's ends read and write different buffers.
// One tile = block `bid` of the RVE's local grid (L.local_blocks blocks).  FIRST
// is a run-time flag (not a template parameter) so that the local step compiles
// to one instruction sequence for both entry paths: a solve resumed from a saved
// state then reproduces the uninterrupted run bit for bit.
template <typename T, int D, int MODEL, bool WRITE_R, bool DU, bool CF>
__device__ __forceinline__ void local_tile(const Launch& L, int bid, const bool FIRST_ARG, int only_if_rho_changed) {
    constexpr int NN = D * D;
    Ctrl* __restrict__ ctrl = L.ctrl;
    double* __restrict__ hist = L.hist;
    double* __restrict__ partials = L.partials;
    T* F0 = Set<T>::F(L, 0);
    T* F1 = Set<T>::F(L, 1);
    T* Lam = Set<T>::Lm(L);
    const T* U0 = Set<T>::U(L, 0);
    const T* U1 = Set<T>::U(L, 1);
    const uint8_t* __restrict__ phase = L.phase;
    const T* __restrict__ mat = Set<T>::mat(L);
    const int nparam = L.nparam;
    const int n = L.n;
    const long long V = L.V;
    float* __restrict__ Rout = L.R32;
    const float* __restrict__ DUin = L.D32;
    const Dirs<T> dir = Set<T>::dirs(L);
    const int nblk = L.local_blocks;
    __shared__ int s_hist[kNewtonBins];       // fraction-converged local steps

    // the increment form needs the previous iteration's R: never the first step of a run
    constexpr bool INC = WRITE_R && DU && !is_lce(MODEL) && std::is_same<T, double>::value;
    if (INC && FIRST_ARG) return;
    const bool FIRST = INC ? false : FIRST_ARG;
    if (ctrl->done) return;
    if (FIRST && only_if_rho_changed && !ctrl->rho_changed) return;
    const long long k = ctrl->k;
    const int par = (int)(k & 1);
    T *Fcur, *Fnext;
    const T *Unew, *Uold;
    if (FIRST) {
        Fcur = par ? F1 : F0;
        Fnext = par ? F0 : F1;
        Unew = par ? U1 : U0;
        Uold = nullptr;
    } else {
        Fcur = par ? F0 : F1;
        Fnext = par ? F1 : F0;
        Unew = par ? U0 : U1;
        Uold = par ? U1 : U0;
    }
    const T rho = (T)ctrl->rho;
    const T half_n = Set<T>::half_n(L);
    const T two_nsq = Set<T>::two_nsq(L);
    const float half_n32 = L.half_n32;
    // double-word polish: F_{k+1} in buffer k & 1 (see above), rho split once
    float* Fc_dw = reinterpret_cast<float*>(par ? F1 : F0);
    float* Fn_dw = reinterpret_cast<float*>(par ? F0 : F1);
    const dw rho_dw = INC ? dw_from(ctrl->rho) : dw{0.f, 0.f};
    // deviation form of the polish: Z = W_F(F_hi) - Lambda_hi per voxel in the idle double
    // Lambda buffer, formed on the polish's first step
    float* Zlin = reinterpret_cast<float*>(L.L64);
    const bool z_fresh = INC && !ctrl->z_valid;
    const int cap = ctrl->newton_cap;
    const T ntol = (T)ctrl->newton_tol;
    // inexact local steps (Section 2.1): |grad phi| <= f mu_ref r_d, with r_d of the
    // last completed check (a redone step uses the same value as the pass it
    // replaces); the first local step of a solve is exact
    const double rd_use = FIRST ? (only_if_rho_changed ? ctrl->rd_local : 0.0) : ctrl->r_d;
    const T gtol = INC ? T(0) : (T)(ctrl->local_ratio * ctrl->mu_ref * rd_use);
    // CF: the float neo-Hookean law in 3D with exact local steps (no member of the launch
    // takes approximate ones) solves Step 1 in closed form (nh3_closed_form)
    constexpr bool kClosedForm = CF;
    static_assert(!CF || (std::is_same<T, float>::value && D == 3 && MODEL == kNeoHooke && !WRITE_R && !DU),
                  "closed-form local step: float neo-Hookean law in 3D only");
    // G_{k+1} - G_k = (<F>_{k+1} - <F>_k) + D(u~_{k+1} - u~_k); the uniform first
    // term (nonzero only under mixed control) enters the voxel sums of r_d in closed
    // form in the last block (D u~ sums to zero over the cell), except in the
    // increment form, where it is part of e voxel by voxel
    T Fb[NN];
    float dFb[NN];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            Fb[i * D + j] = (T)ctrl->Fbar[i * 3 + j];
            dFb[i * D + j] = INC ? (float)(ctrl->Fbar[i * 3 + j] - ctrl->Fbar_prev[i * 3 + j]) : 0.f;
        }

    // per-thread residual sums: float in the float kernels and in the increment form
    // (whose terms are float; tens of voxels per thread keep the relative error of the
    // sums near 1e-6, ample for the tolerance tests), double otherwise; the block and
    // grid sums are always double
    using Acc = typename std::conditional<sizeof(T) == 4 || INC, float, double>::type;
    // Section 4.2's first strategy (fraction-converged local steps): this pass's
    // histogram of Newton counts sets the next pass's cap (one pass of lag, no barrier)
    const bool frac_on = !INC && !FIRST && !is_lce(MODEL) && ctrl->local_fraction > 0.0;
    if (frac_on) {
        if (threadIdx.x < kNewtonBins) s_hist[threadIdx.x] = 0;
        __syncthreads();
    }
    Acc rp2a = Acc(0), rd2a = Acc(0), rl2a = Acc(0);
    int nmax = 0, nfail = 0;
    const int chunk = L.local_chunk;
    const FastDiv dn = L.plan.div_n;
    for (long long v = bid * (long long)chunk + threadIdx.x; threadIdx.x < chunk && v < V; v += (long long)nblk * chunk) {
        const Nbr<D> nb = neighbours<D>((int)v, dn);
        if constexpr (INC) {
            float dG[NN], spf, sdf;
            grad_u<float, D>(DUin, V, nb, dFb, half_n32, dG);
            const int ph = phase[v];
            const dw mu{__ldg(L.mat32 + ph * nparam), __ldg(L.mat32lo + ph * nparam)};
            const dw lam{__ldg(L.mat32 + ph * nparam + 1), __ldg(L.mat32lo + ph * nparam + 1)};
            bool conv;
            polish_voxel_dev<D, MODEL>(Fc_dw, Fn_dw, L.LH32, L.LL32, Zlin, Rout, dG, mu, lam, rho_dw.hi, z_fresh, v,
                                       V, spf, sdf, conv);
            rp2a += spf;
            rd2a += sdf;
            nmax = max(nmax, 1);
            nfail += conv ? 0 : 1;
            continue;
        }
        T G[NN], L[NN], F[NN];
        grad_u<T, D>(Unew, V, nb, Fb, half_n, G);
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            L[p] = Lam[p * V + v];
            F[p] = Fcur[p * V + v];
        }
        if (!FIRST) {
            // squares are summed per voxel in T (9 terms) and the voxel sums in double
            T sp = T(0), sd = T(0);
#pragma unroll
            for (int p = 0; p < NN; ++p) {
                const T df = G[p] - F[p];
                L[p] += rho * df;
                sp += df * df;
                Lam[p * V + v] = L[p];
            }
            if constexpr (DU) {
                const float zero[NN] = {};
                float dG[NN];
                grad_u<float, D>(DUin, V, nb, zero, half_n32, dG);
                float sdf = 0.f;
#pragma unroll
                for (int p = 0; p < NN; ++p) sdf += dG[p] * dG[p];
                sd = (T)sdf;
            } else {
                T Go[NN];
                grad_u<T, D>(Uold, V, nb, Fb, half_n, Go);
#pragma unroll
                for (int p = 0; p < NN; ++p) {
                    const T dg = G[p] - Go[p];
                    sd += dg * dg;
                }
            }
            rp2a += (Acc)sp;
            rd2a += (Acc)sd;
        }
        bool conv;
        int it;
        T B[NN];
#pragma unroll
        for (int p = 0; p < NN; ++p) B[p] = L[p] + rho * G[p];
        if constexpr (is_lce(MODEL)) {
            // director of the current iterate (same parity as F) and the explicit Frank force
            const T* nCur = FIRST ? (par ? dir.N1 : dir.N0) : (par ? dir.N0 : dir.N1);
            T* nNext = FIRST ? (par ? dir.N0 : dir.N1) : (par ? dir.N1 : dir.N0);
            const T* q = mat + phase[v] * nparam;
            const T kf = __ldg(q + 4) * two_nsq;
            // dissipation of one time step (Section 5.1): cF/2 |F - Fprev|^2 adds cF to the
            // penalty and cF Fprev to B; on |n| = 1, cn/2 |n - nprev|^2 is -cn n.nprev + const,
            // a force cn nprev next to the explicit Frank force
            const T cF = __ldg(q + 8), cn = __ldg(q + 9);
            T nv[3], fr[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T* c = nCur + i * V;
                nv[i] = c[v];
                fr[i] = kf * (c[nb.xp] + c[nb.xm] + c[nb.yp] + c[nb.ym] + c[nb.zp] + c[nb.zm]) + cn * dir.np[i * V + v];
            }
#pragma unroll
            for (int p = 0; p < NN; ++p) B[p] += cF * dir.Fp[p * V + v];
            const Lce<T> m = load_lce<T, MODEL == kLceInc>(phase, mat, nparam, v, dir.ref, V);
            T gn2 = T(0);
            if constexpr (MODEL == kLceInc)  // always solved to the step tolerance (no gradient stop)
                it = newton_lce_inc<T>(m, F, nv, B, fr, rho + cF, rho, cap, ntol, conv);
            else
                it = newton_lce<T>(m, F, nv, B, fr, rho + cF, cap, ntol, conv, gtol, &gn2);
            rl2a += (Acc)gn2;
#pragma unroll
            for (int i = 0; i < 3; ++i) nNext[i * V + v] = nv[i];
        } else {
            using Law = typename LawOf<T, D, MODEL>::type;
            const Law m = load_law<Law, T>(phase, mat, nparam, v);
            T gn2 = T(0);
            if constexpr (kClosedForm) {
                if (nh3_closed_form(m.mu, m.lam, rho, B, det<T, 3>(F), F)) {
                    it = 1;
                    conv = true;
                } else {
                    it = steepest_descent<T, 3>(m, F, B, rho, cap, ntol, conv);
                }
            } else {
                it = newton<T, D>(m, F, B, rho, cap, ntol, conv, gtol, &gn2);
            }
            rl2a += (Acc)gn2;
        }
        nmax = max(nmax, it);
        nfail += conv ? 0 : 1;
        // Every Newton step keeps J > 0, so J <= 0 after the local step means the voxel
        // started inverted (a state or <F> with det <= 0) and W is undefined there: the
        // residual sum is made NaN, which ends the solve with RVE_E_NUMERICAL.
        if (!conv && !(det<T, D>(F) > T(0))) rp2a = Acc(NAN);
        if (frac_on && conv) atomicAdd(&s_hist[min(max(it + 1, 2) / 2, kNewtonBins) - 1], 1);
#pragma unroll
        for (int p = 0; p < NN; ++p) Fnext[p * V + v] = F[p];
        if constexpr (WRITE_R) {
#pragma unroll
            for (int p = 0; p < NN; ++p) Rout[p * V + v] = (float)(F[p] - G[p]);
        }
    }
    if (FIRST) return;
    finish_pass<D, INC, Acc>(ctrl, hist, partials, bid, nblk, V, k, rp2a, rd2a, rl2a, nmax, nfail, frac_on, s_hist);
}


// Resident blocks per SM the register budget is cut for: the float elastic laws
// are latency-bound at fewer.
constexpr int kCfMinBlocks = 6;  // 80 registers: two whole waves of the 1824-block grid
template <typename T, int MODEL, bool WRITE_R, bool DU, bool CF>
constexpr int local_min_blocks() {
    if (is_lce(MODEL)) return 1;
    if (CF) return kCfMinBlocks;
    if (sizeof(T) == 4) return 4;
    return (WRITE_R && DU) ? 4 : 1;  // the polish: FP32 work; 3, 5, 6 blocks measured slower
}

template <typename T, int D, int MODEL, bool WRITE_R, bool DU, bool CF = false>
__global__ void __launch_bounds__(kLocalThreads, local_min_blocks<T, MODEL, WRITE_R, DU, CF>())
k_local(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles, int first,
        int only_if_rho_changed) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        local_tile<T, D, MODEL, WRITE_R, DU, CF>(rds[tl.x], tl.y, first != 0, only_if_rho_changed);
        __syncthreads();
    }
}

// Periodic neighbours of voxel v on an N^3 grid: by shifts and masks for a compile-time
// N (a power of two), by the multiply-high divisor of the run-time n for N = 0.
template <int N>
__device__ __forceinline__ Nbr<3> nbr3(int v, const FastDiv& dn) {
    if constexpr (N == 0) {
        return neighbours<3>(v, dn);
    } else {
        constexpr int LOG = N == 128 ? 7 : (N == 256 ? 8 : 9);
        static_assert(N == (1 << LOG), "power-of-two grids");
        const int x = v & (N - 1), y = (v >> LOG) & (N - 1), z = v >> (2 * LOG);
        Nbr<3> o;
        o.xp = v + (x == N - 1 ? 1 - N : 1);
        o.xm = v + (x == 0 ? N - 1 : -1);
        o.yp = v + (y == N - 1 ? (1 - N) * N : N);
        o.ym = v + (y == 0 ? (N - 1) * N : -N);
        o.zp = v + (z == N - 1 ? (1 - N) * N * N : N * N);
        o.zm = v + (z == 0 ? (N - 1) * N * N : -N * N);
        return o;
    }
}

// The fused pass of one RVE for the float neo-Hookean law in 3D with exact local steps
// (closed-form Step 1) on an N^3 grid, N = 128, 256 or 512, or N = 0: any other grid of
// at least 1824 x 128 voxels (a full local grid; the run-time n and V come in the args): the same steps, sums and
// tile partials as local_tile's closed-form instance, arranged so that the voxel loop
// keeps few values in registers.  The RVE's buffers and constants are kernel parameters
// (read from the constant bank where they are used), the grid size is a compile-time
// constant (neighbours by shifts and masks, 32-bit offsets: 9 N^3 < 2^31), Fbar is read
// from shared memory, and the previous iterate F_{k+1} is not held through the local
// solve (its rare fallback reloads it).  local_tile's instance keeps the RVE descriptor
// of each tile in registers and spills at the register cap of 6 blocks per SM (at 128^3:
// 133 us per launch there, 108 us here).  F and Lambda are read and written with
// evict-first hints (each value is touched once per pass), which leaves L1 and L2 to the
// u~ stencils.
struct CfArgs {
    Ctrl* ctrl;
    double* hist;
    double* partials;
    float* F[2];
    float* Lam;
    const float* U[2];
    const uint8_t* phase;
    const float* mat;
    int nparam;
    int nblk;    // tiles of the RVE's local grid
    int chunk;   // voxels of a tile per sweep
    float half_n;
    const double* zpart;  // the z pass's tile sums for r_d (Launch::Sprev), or null
    int nz;
    int V;                // voxels and the multiply-high divisor of n (N = 0 only)
    FastDiv dn;
};

template <int N>
__global__ void __launch_bounds__(kLocalThreads, kCfMinBlocks)
k_local_cf(const __grid_constant__ CfArgs a, int first, int only_if_rho_changed) {
    static_assert(N == 0 || N == 128 || N == 256 || N == 512, "fixed grid sizes or run-time (0)");
    const int V = N ? N * N * N : a.V;
    constexpr int NN = 9;
    __shared__ float s_fb[NN];
    Ctrl* __restrict__ ctrl = a.ctrl;
    const bool FIRST = first != 0;
    if (ctrl->done) return;
    if (FIRST && only_if_rho_changed && !ctrl->rho_changed) return;
    const long long k = ctrl->k;
    // buffers as in local_tile: F_{k+1}, u~_{k+1} in buffer (k + 1) & 1 for the fused
    // pass, F_k, u~_k in buffer k & 1 for the local step alone
    const bool q = FIRST ? !(k & 1) : (k & 1);
    const float* __restrict__ Fcur = q ? a.F[0] : a.F[1];
    float* __restrict__ Fnext = q ? a.F[1] : a.F[0];
    const float* __restrict__ Unew = q ? a.U[0] : a.U[1];
    const float* __restrict__ Uold = q ? a.U[1] : a.U[0];
    const float rho = (float)ctrl->rho;
    const int cap = ctrl->newton_cap;
    const float ntol = (float)ctrl->newton_tol;
    // r_d from the z pass of this iteration when it summed the spectral change, else from
    // the u~_k stencil here
    const bool spec = !FIRST && a.zpart && ctrl->spec_sum;
    if (threadIdx.x < NN) s_fb[threadIdx.x] = (float)ctrl->Fbar[(threadIdx.x / 3) * 3 + threadIdx.x % 3];
    __syncthreads();
    const volatile float* Fb = s_fb;
    const float hn = a.half_n;
    for (int t = blockIdx.x; t < a.nblk; t += gridDim.x) {
        float rp2a = 0.f, rd2a = 0.f;
        int nmax = 0, nfail = 0;
        for (int v = t * a.chunk + threadIdx.x; threadIdx.x < a.chunk && v < V; v += a.nblk * a.chunk) {
            const Nbr<3> nb = nbr3<N>(v, a.dn);
            const int xp = nb.xp, xm = nb.xm, yp = nb.yp, ym = nb.ym, zp = nb.zp, zm = nb.zm;
            float G[NN], L[NN], F[NN];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float* u = Unew + i * V;
                G[3 * i + 0] = Fb[3 * i + 0] + (__ldg(u + xp) - __ldg(u + xm)) * hn;
                G[3 * i + 1] = Fb[3 * i + 1] + (__ldg(u + yp) - __ldg(u + ym)) * hn;
                G[3 * i + 2] = Fb[3 * i + 2] + (__ldg(u + zp) - __ldg(u + zm)) * hn;
            }
#pragma unroll
            for (int p = 0; p < NN; ++p) {
                L[p] = __ldcs(a.Lam + p * V + v);
                F[p] = __ldcs(Fcur + p * V + v);
            }
            // the phase byte is read before the stores below: a byte load may alias them and
            // would otherwise wait for them
            const NeoHooke<float, 3> m = load_law<NeoHooke<float, 3>, float>(a.phase, a.mat, a.nparam, v);
            const float J0 = det<float, 3>(F);
            if (!FIRST) {
                // Steps 3-4 of iteration k (voxel sums in float, tile sums in double)
                float sp = 0.f, sd = 0.f;
#pragma unroll
                for (int p = 0; p < NN; ++p) {
                    const float df = G[p] - F[p];
                    L[p] += rho * df;
                    sp += df * df;
                    __stcs(a.Lam + p * V + v, L[p]);
                }
                if (!spec) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float* u = Uold + i * V;
                        const float g0 = Fb[3 * i + 0] + (__ldg(u + xp) - __ldg(u + xm)) * hn;
                        const float g1 = Fb[3 * i + 1] + (__ldg(u + yp) - __ldg(u + ym)) * hn;
                        const float g2 = Fb[3 * i + 2] + (__ldg(u + zp) - __ldg(u + zm)) * hn;
                        const float d0 = G[3 * i + 0] - g0, d1 = G[3 * i + 1] - g1, d2 = G[3 * i + 2] - g2;
                        sd += d0 * d0;
                        sd += d1 * d1;
                        sd += d2 * d2;
                    }
                }
                rp2a += sp;
                rd2a += sd;
            }
            float B[NN];
#pragma unroll
            for (int p = 0; p < NN; ++p) B[p] = L[p] + rho * G[p];
            float Fo[NN];
            int it = 1;
            bool conv = true;
            if (!nh3_closed_form(m.mu, m.lam, rho, B, J0, Fo)) {
#pragma unroll
                for (int p = 0; p < NN; ++p) Fo[p] = __ldg(Fcur + p * V + v);
                it = steepest_descent<float, 3>(m, Fo, B, rho, cap, ntol, conv);
            }
            nmax = max(nmax, it);
            nfail += conv ? 0 : 1;
            // as in local_tile: J <= 0 after the local step means an inverted start
            if (!conv && !(det<float, 3>(Fo) > 0.f)) rp2a = NAN;
#pragma unroll
            for (int p = 0; p < NN; ++p) __stcs(Fnext + p * V + v, Fo[p]);
        }
        if (!FIRST)
            finish_pass<3, false, float>(ctrl, a.hist, a.partials, t, a.nblk, (long long)V, k, rp2a, rd2a, 0.f, nmax,
                                         nfail, false, nullptr, spec, a.zpart, a.nz);
        __syncthreads();
    }
}

// The double-word polish step (local_tile's increment form, polish_voxel_dev) of one RVE
// of an elastic law in 3D on an N^3 grid, N = 128, 256 or 512 or run-time (0), laid out
// like k_local_cf: buffers and constants as kernel parameters, N fixed at compile time,
// 32-bit offsets.  Same arithmetic and tile partials as the tile-table instance.
struct PolishArgs {
    Ctrl* ctrl;
    double* hist;
    double* partials;
    float* F[2];       // the double F buffers holding (hi, lo) float pairs
    float* Lhi;
    float* Llo;
    float* Z;          // the idle double Lambda buffer
    float* R;          // R = F_{k+2} - G_{k+1}, read and rewritten
    const float* DU;   // float u~ increment of the last increment projection
    const uint8_t* phase;
    const float* mat;
    const float* mat_lo;
    int nparam;
    int nblk;
    int chunk;
    float half_n;
    int V;             // voxels and the multiply-high divisor of n (N = 0 only)
    FastDiv dn;
};

template <int N, int MODEL>
__global__ void __launch_bounds__(kLocalThreads, 4) k_polish_fixed(const __grid_constant__ PolishArgs a) {
    static_assert(N == 0 || N == 128 || N == 256 || N == 512, "fixed grid sizes or run-time (0)");
    const int V = N ? N * N * N : a.V;
    constexpr int NN = 9;
    __shared__ float s_dfb[NN];
    Ctrl* __restrict__ ctrl = a.ctrl;
    if (ctrl->done) return;
    const long long k = ctrl->k;
    // F_{k+1} in buffer k & 1 (see local_tile)
    float* Fc = (k & 1) ? a.F[1] : a.F[0];
    float* Fn = (k & 1) ? a.F[0] : a.F[1];
    const float rho = dw_from(ctrl->rho).hi;
    const bool z_fresh = !ctrl->z_valid;
    if (threadIdx.x < NN) {
        const int i = threadIdx.x / 3, j = threadIdx.x % 3;
        s_dfb[threadIdx.x] = (float)(ctrl->Fbar[i * 3 + j] - ctrl->Fbar_prev[i * 3 + j]);
    }
    __syncthreads();
    const volatile float* dFb = s_dfb;
    const float hn = a.half_n;
    for (int t = blockIdx.x; t < a.nblk; t += gridDim.x) {
        float rp2a = 0.f, rd2a = 0.f;
        int nmax = 0, nfail = 0;
        for (int v = t * a.chunk + threadIdx.x; threadIdx.x < a.chunk && v < V; v += a.nblk * a.chunk) {
            const Nbr<3> nb = nbr3<N>(v, a.dn);
            const int xp = nb.xp, xm = nb.xm, yp = nb.yp, ym = nb.ym, zp = nb.zp, zm = nb.zm;
            float dG[NN], spf, sdf;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float* u = a.DU + i * V;
                dG[3 * i + 0] = dFb[3 * i + 0] + (__ldg(u + xp) - __ldg(u + xm)) * hn;
                dG[3 * i + 1] = dFb[3 * i + 1] + (__ldg(u + yp) - __ldg(u + ym)) * hn;
                dG[3 * i + 2] = dFb[3 * i + 2] + (__ldg(u + zp) - __ldg(u + zm)) * hn;
            }
            const int ph = a.phase[v];
            const dw mu{__ldg(a.mat + ph * a.nparam), __ldg(a.mat_lo + ph * a.nparam)};
            const dw lam{__ldg(a.mat + ph * a.nparam + 1), __ldg(a.mat_lo + ph * a.nparam + 1)};
            bool conv;
            polish_voxel_dev<3, MODEL, int>(Fc, Fn, a.Lhi, a.Llo, a.Z, a.R, dG, mu, lam, rho, z_fresh, v, V, spf, sdf,
                                            conv);
            rp2a += spf;
            rd2a += sdf;
            nmax = 1;
            nfail += conv ? 0 : 1;
        }
        finish_pass<3, true, float>(ctrl, a.hist, a.partials, t, a.nblk, (long long)V, k, rp2a, rd2a, 0.f, nmax,
                                    nfail, false, nullptr);
        __syncthreads();
    }
}

// Mixed macroscopic control (Section 2.3; the UNI, PE and EB protocols of Section
// 5.3).  The free components of <F> join Step 2's minimisation of
// |<F> + D u~ - Q|^2, Q = F_{k+1} - Lambda_k / rho; D u~ has zero mean, so their
// minimiser is <Q>.  Runs before the iteration's projection, with ctrl->k = k;
// keeps the previous <F> for r_d.  Sums in double with the fixed-order scheme.
// DWS: the double polish's double-word state (F_{k+1} in F buffer k & 1, Lambda in
// Lh, Ll), read through T = float pointers.
template <typename T, int D, bool DWS>
__global__ void __launch_bounds__(kLocalThreads)
k_macro(Ctrl* __restrict__ ctrl, double* __restrict__ partials, const T* F0, const T* F1, const T* Lam,
        const float* __restrict__ Lh, const float* __restrict__ Ll, long long V) {
    constexpr int NN = D * D;
    __shared__ double s_sum[kLocalThreads / 32][2 * NN];
    __shared__ int s_last;
    if (ctrl->done) return;
    const T* F = ((ctrl->k & 1) != 0) != DWS ? F0 : F1;  // F_{k+1}
    double acc[2 * NN];
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) acc[p] = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            if constexpr (DWS) {
                acc[p] += (double)F[p * V + v] + (double)F[(NN + p) * V + v];
                acc[NN + p] += (double)Lh[p * V + v] + (double)Ll[p * V + v];
            } else {
                acc[p] += (double)F[p * V + v];
                acc[NN + p] += (double)Lam[p * V + v];
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) {
        const double s = warp_sum(acc[p]);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* pp = partials + (size_t)blockIdx.x * kPartialStride;
        for (int p = 0; p < 2 * NN; ++p) {
            double s = 0;
            for (int w = 0; w < kLocalThreads / 32; ++w) s += s_sum[w][p];
            pp[p] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->counter2, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) acc[p] = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const double* pp = partials + (size_t)i * kPartialStride;
#pragma unroll
        for (int p = 0; p < 2 * NN; ++p) acc[p] += __ldcg(pp + p);
    }
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) {
        const double s = warp_sum(acc[p]);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    Ctrl* c = ctrl;
    for (int i = 0; i < 9; ++i) c->Fbar_prev[i] = c->Fbar[i];
    for (int p = 0; p < NN; ++p) {
        const int i = p / D, j = p % D;
        if (!((c->free_mask >> (3 * i + j)) & 1u)) continue;
        double sf = 0, sl = 0;
        for (int w = 0; w < kLocalThreads / 32; ++w) {
            sf += s_sum[w][p];
            sl += s_sum[w][NN + p];
        }
        c->Fbar[3 * i + j] = sf / (double)V - (sl / (double)V) * c->inv_rho;
    }
    c->counter2 = 0u;
}

// <W_F(F_k)> and <Lambda_k>, summed in double with the same fixed-order scheme.
template <typename T, int D, int MODEL>
__global__ void __launch_bounds__(kLocalThreads)
k_stress(Ctrl* __restrict__ ctrl, double* __restrict__ partials, const T* F0, const T* F1, const T* Lam,
         const uint8_t* __restrict__ phase, const T* __restrict__ mat, int nparam, long long V, Dirs<T> dir) {
    constexpr int NN = D * D;
    __shared__ double s_sum[kLocalThreads / 32][2 * NN];
    __shared__ int s_last;
    const T* F = (ctrl->k & 1) ? F1 : F0;
    double acc[2 * NN];
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) acc[p] = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        T Fv[NN], P[NN];
#pragma unroll
        for (int p = 0; p < NN; ++p) Fv[p] = F[p * V + v];
        if constexpr (MODEL == kLceInc) {
            // the reaction pressure is not part of the state: Lambda stands for the stress
#pragma unroll
            for (int p = 0; p < NN; ++p) P[p] = Lam[p * V + v];
        } else if constexpr (MODEL == kLce) {
            const T* Nk = (ctrl->k & 1) ? dir.N1 : dir.N0;
            const T nv[3] = {Nk[v], Nk[V + v], Nk[2 * V + v]};
            load_lce<T>(phase, mat, nparam, v, dir.ref, V).stress(Fv, nv, P);
            const T cF = __ldg(mat + phase[v] * nparam + 8);  // with the viscous stress cF (F - Fprev)
#pragma unroll
            for (int p = 0; p < NN; ++p) P[p] += cF * (Fv[p] - dir.Fp[p * V + v]);
        } else {
            using Law = typename LawOf<T, D, MODEL>::type;
            const Law m = load_law<Law, T>(phase, mat, nparam, v);
            m.stress(Fv, P);
        }
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            acc[p] += (double)P[p];
            acc[NN + p] += (double)Lam[p * V + v];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) {
        const double s = warp_sum(acc[p]);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double* pp = partials + (size_t)blockIdx.x * kPartialStride;
        for (int p = 0; p < 2 * NN; ++p) {
            double s = 0;
            for (int w = 0; w < kLocalThreads / 32; ++w) s += s_sum[w][p];
            pp[p] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(&ctrl->counter2, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) acc[p] = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        const double* pp = partials + (size_t)i * kPartialStride;
#pragma unroll
        for (int p = 0; p < 2 * NN; ++p) acc[p] += __ldcg(pp + p);
    }
#pragma unroll
    for (int p = 0; p < 2 * NN; ++p) {
        const double s = warp_sum(acc[p]);
        if (lane == 0) s_sum[warp][p] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 0; i < 9; ++i) {
        ctrl->stress[i] = 0.0;
        ctrl->lam_mean[i] = 0.0;
    }
    for (int p = 0; p < NN; ++p) {
        double s = 0, l = 0;
        for (int w = 0; w < kLocalThreads / 32; ++w) {
            s += s_sum[w][p];
            l += s_sum[w][NN + p];
        }
        const int i = p / D, j = p % D;
        ctrl->stress[i * 3 + j] = s / (double)V;
        ctrl->lam_mean[i * 3 + j] = l / (double)V;
    }
    ctrl->counter2 = 0u;
}

// Copy the current state (F_k, Lambda_k, u~_k) between the float and double sets.
template <typename S, typename Dd>
__global__ void k_convert(const Ctrl* __restrict__ ctrl, const S* Fs0, const S* Fs1, const S* Ls, const S* Us0,
                          const S* Us1, Dd* Fd0, Dd* Fd1, Dd* Ld, Dd* Ud0, Dd* Ud1, long long nF, long long nU,
                          const S* Ns0, const S* Ns1, Dd* Nd0, Dd* Nd1, long long nN) {
    const int par = (int)(ctrl->k & 1);
    const S* Fs = par ? Fs1 : Fs0;
    const S* Us = par ? Us1 : Us0;
    const S* Ns = par ? Ns1 : Ns0;
    Dd* Fd = par ? Fd1 : Fd0;
    Dd* Ud = par ? Ud1 : Ud0;
    Dd* Nd = par ? Nd1 : Nd0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nF; i += (long long)gridDim.x * blockDim.x) {
        Fd[i] = (Dd)Fs[i];
        Ld[i] = (Dd)Ls[i];
        if (i < nU) Ud[i] = (Dd)Us[i];
        if (i < nN) Nd[i] = (Dd)Ns[i];
    }
}

// ------------------------------------------------------------------ dispatch

template <typename T, int D, int MODEL>
cudaError_t run_init(const Launch& L, bool lambda_zero) {
    k_init<T, D, MODEL><<<L.local_blocks, kLocalThreads, 0, L.stream>>>(
        L.ctrl, Set<T>::F(L, 0), Set<T>::F(L, 1), Set<T>::Lm(L), Set<T>::U(L, 0), Set<T>::U(L, 1), L.phase, Set<T>::mat(L),
        L.nparam, L.V, lambda_zero ? 1 : 0, Set<T>::dirs(L));
    return cudaGetLastError();
}

}  // namespace

// Whether a member's fused local pass runs the lean per-RVE kernel (k_local_cf in the
// float phase, k_polish_fixed in the double-word polish): 3D, the neo-Hookean law with
// exact local steps (float phase) or an elastic law (polish), and a grid of N = 128, 256,
// 512 or a full local grid (every tile a whole block of voxels), so that a launch of its
// own fills the GPU.  A function of the member alone: its results are the same in any batch.
bool lean_local(const Launch& L, bool exact, bool polish) {
    if (L.dim != 3) return false;
    if (polish ? !(L.model == kNeoHooke || L.model == kLinear) : !(L.model == kNeoHooke && exact)) return false;
    if (L.n == 128 || L.n == 256 || L.n == 512) return true;
    return L.local_blocks == kLocalTileCap && L.local_chunk == kLocalThreads;
}

namespace {

// mode: 0 plain, 1 write R (first polish iteration), 2 write R and read the float u~ increment
template <typename T, int D, int MODEL>
cudaError_t run_local(const Exec& E, bool first, bool only_if, int mode) {
    const int nt = E.ntiles[kTilesLocal];
    const int2* tl = E.tiles[kTilesLocal];
    auto go = [&](auto kern, int is_first, int flag) {
        const int grid = persistent_grid((const void*)kern, kLocalThreads, 0, nt);
        kern<<<grid, kLocalThreads, 0, E.stream>>>(E.rds, tl, nt, is_first, flag);
    };
    // Members with a lean kernel (lean_local) run one launch each; the others' tiles come
    // first in the local tile table (the engine orders them so) and share one tile launch.
    // Returns false when no member has a lean kernel.
    auto lean_split = [&](bool polish, auto&& lean_launch, auto&& tile_launch) {
        if (E.nmem <= 0) return false;
        int prefix = 0;
        bool any = false, exact_pre = true;
        for (int i = 0; i < E.nmem; ++i) {
            if (lean_local(*E.mem[i], E.mem_exact[i] != 0, polish)) {
                any = true;
            } else {
                prefix += tiles_local(*E.mem[i]);
                exact_pre = exact_pre && E.mem_exact[i];
            }
        }
        if (!any) return false;
        bool ordered = true;  // the non-lean members' tiles form the prefix
        for (int i = 0; i < E.nmem; ++i)
            if (!lean_local(*E.mem[i], E.mem_exact[i] != 0, polish) &&
                E.mem_tile0[i] + tiles_local(*E.mem[i]) > prefix)
                ordered = false;
        if (ordered) {
            if (prefix > 0) tile_launch(0, prefix, exact_pre);
        } else {
            for (int i = 0; i < E.nmem; ++i)
                if (!lean_local(*E.mem[i], E.mem_exact[i] != 0, polish))
                    tile_launch(E.mem_tile0[i], tiles_local(*E.mem[i]), E.mem_exact[i] != 0);
        }
        for (int i = 0; i < E.nmem; ++i)
            if (lean_local(*E.mem[i], E.mem_exact[i] != 0, polish)) lean_launch(*E.mem[i]);
        return true;
    };
    auto tile_range = [&](auto kern, int t0, int cnt, int is_first, int flag) {
        const int grid = persistent_grid((const void*)kern, kLocalThreads, 0, cnt);
        kern<<<grid, kLocalThreads, 0, E.stream>>>(E.rds, tl + t0, cnt, is_first, flag);
    };
    if constexpr (std::is_same<T, float>::value && D == 3 && MODEL == kNeoHooke) {
        const int f = first ? 1 : 0, fo = first && only_if ? 1 : 0;
        const bool split = lean_split(
            false,
            [&](const Launch& M) {
                CfArgs a{M.ctrl,     M.hist,           M.partials,       {M.F32[0], M.F32[1]},
                         M.L32,      {M.U32[0], M.U32[1]}, M.phase,      M.mat32,
                         M.nparam,   M.local_blocks,   M.local_chunk,    M.half_n32,
                         M.zpart,    M.nz,             (int)M.V,         M.plan.div_n};
                auto lean = [&](auto kern) {
                    const int grid = persistent_grid((const void*)kern, kLocalThreads, 0, M.local_blocks);
                    kern<<<grid, kLocalThreads, 0, E.stream>>>(a, f, fo);
                };
                if (M.n == 128) lean(k_local_cf<128>);
                else if (M.n == 256) lean(k_local_cf<256>);
                else if (M.n == 512) lean(k_local_cf<512>);
                else lean(k_local_cf<0>);
            },
            [&](int t0, int cnt, bool exact) {
                if (exact) tile_range(k_local<T, D, MODEL, false, false, true>, t0, cnt, f, fo);
                else tile_range(k_local<T, D, MODEL, false, false>, t0, cnt, f, fo);
            });
        if (split) return cudaGetLastError();
        if (E.exact_local) {
            go(k_local<T, D, MODEL, false, false, true>, first ? 1 : 0, first && only_if ? 1 : 0);
            return cudaGetLastError();
        }
    }
    if (first) {
        go(k_local<T, D, MODEL, false, false>, 1, only_if ? 1 : 0);
        return cudaGetLastError();
    }
    if constexpr (std::is_same<T, double>::value && D == 3 && (MODEL == kNeoHooke || MODEL == kLinear)) {
        if (mode == 2) {
            const bool split = lean_split(
                true,
                [&](const Launch& M) {
                    PolishArgs a{M.ctrl, M.hist, M.partials,
                                 {reinterpret_cast<float*>(M.F64[0]), reinterpret_cast<float*>(M.F64[1])},
                                 M.LH32, M.LL32, reinterpret_cast<float*>(M.L64), M.R32, M.D32, M.phase, M.mat32,
                                 M.mat32lo, M.nparam, M.local_blocks, M.local_chunk, M.half_n32, (int)M.V,
                                 M.plan.div_n};
                    auto lean = [&](auto kern) {
                        const int grid = persistent_grid((const void*)kern, kLocalThreads, 0, M.local_blocks);
                        kern<<<grid, kLocalThreads, 0, E.stream>>>(a);
                    };
                    if (M.n == 128) lean(k_polish_fixed<128, MODEL>);
                    else if (M.n == 256) lean(k_polish_fixed<256, MODEL>);
                    else if (M.n == 512) lean(k_polish_fixed<512, MODEL>);
                    else lean(k_polish_fixed<0, MODEL>);
                },
                [&](int t0, int cnt, bool) { tile_range(k_local<T, D, MODEL, true, true>, t0, cnt, 0, 0); });
            if (split) return cudaGetLastError();
        }
    }
    if constexpr (std::is_same<T, double>::value) {
        if (mode == 1) {
            go(k_local<T, D, MODEL, true, false>, 0, 0);
            return cudaGetLastError();
        }
        if (mode == 2) {
            go(k_local<T, D, MODEL, true, true>, 0, 0);
            return cudaGetLastError();
        }
    }
    go(k_local<T, D, MODEL, false, false>, 0, 0);
    return cudaGetLastError();
}

template <typename T, int D, int MODEL>
cudaError_t run_stress(const Launch& L) {
    k_stress<T, D, MODEL><<<L.local_blocks, kLocalThreads, 0, L.stream>>>(
        L.ctrl, L.partials, Set<T>::F(L, 0), Set<T>::F(L, 1), Set<T>::Lm(L), L.phase, Set<T>::mat(L), L.nparam, L.V,
        Set<T>::dirs(L));
    return cudaGetLastError();
}

#define RVE_DISPATCH(FN, T, ...)                                                            \
    do {                                                                                    \
        if (L.dim == 2 && L.model == kNeoHooke) return FN<T, 2, kNeoHooke>(__VA_ARGS__);    \
        if (L.dim == 3 && L.model == kNeoHooke) return FN<T, 3, kNeoHooke>(__VA_ARGS__);    \
        if (L.dim == 2 && L.model == kLinear) return FN<T, 2, kLinear>(__VA_ARGS__);        \
        if (L.dim == 3 && L.model == kLinear) return FN<T, 3, kLinear>(__VA_ARGS__);        \
        if (L.dim == 3 && L.model == kLce) return FN<T, 3, kLce>(__VA_ARGS__);              \
        if (L.dim == 3 && L.model == kLceInc) return FN<T, 3, kLceInc>(__VA_ARGS__);        \
        return cudaErrorInvalidValue;                                                       \
    } while (0)

}  // namespace

cudaError_t launch_init(const Launch& L, bool fp64, bool lambda_zero) {
    if (fp64) RVE_DISPATCH(run_init, double, L, lambda_zero);
    RVE_DISPATCH(run_init, float, L, lambda_zero);
}

cudaError_t launch_local(const Exec& E, bool fp64, bool first, bool only_if_rho_changed, int polish_mode) {
    const Launch& L = *E.rep;
    if (fp64) RVE_DISPATCH(run_local, double, E, first, only_if_rho_changed, polish_mode);
    RVE_DISPATCH(run_local, float, E, first, only_if_rho_changed, 0);
}

cudaError_t launch_macro(const Launch& L, bool fp64, cudaStream_t st, bool dws) {
    auto go = [&](auto kern, const auto* F0, const auto* F1, const auto* Lm) {
        kern<<<L.local_blocks, kLocalThreads, 0, st>>>(L.ctrl, L.partials, F0, F1, Lm, L.LH32, L.LL32, L.V);
        return cudaGetLastError();
    };
    if (dws) {
        const float* f0 = reinterpret_cast<const float*>(L.F64[0]);
        const float* f1 = reinterpret_cast<const float*>(L.F64[1]);
        return L.dim == 3 ? go(k_macro<float, 3, true>, f0, f1, L.LH32) : go(k_macro<float, 2, true>, f0, f1, L.LH32);
    }
    if (fp64)
        return L.dim == 3 ? go(k_macro<double, 3, false>, L.F64[0], L.F64[1], L.L64)
                          : go(k_macro<double, 2, false>, L.F64[0], L.F64[1], L.L64);
    return L.dim == 3 ? go(k_macro<float, 3, false>, L.F32[0], L.F32[1], L.L32)
                      : go(k_macro<float, 2, false>, L.F32[0], L.F32[1], L.L32);
}

// float -> double from the IEEE bit fields: exact, like the conversion instruction, with
// integer operations only for zero and normal numbers (exponent rebiased by 1023 - 127,
// fraction shifted up by 52 - 23 bits); subnormal, infinite and NaN inputs take the
// conversion instruction.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long s = (unsigned long long)(u >> 31) << 63;
    if (e - 1u < 254u)
        return __longlong_as_double((long long)(s | ((unsigned long long)(e + 896u) << 52) |
                                                ((unsigned long long)(u & 0x7fffffu) << 29)));
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)s);
    return (double)f;
}

// Double <-> double-word state at the ends of the polish (see local_tile).  With
// k = ctrl->k.  enter (after the polish's first, double iteration, unless the solve
// already stopped): the double F_{k+1} (buffer (k+1) & 1) becomes the double-word
// F_{k+1} in buffer k & 1 and Lambda_k moves to (Lh, Ll).  leave (only after an
// enter): the double-word F_k (buffer (k+1) & 1) becomes the double F_k in buffer
// k & 1 and Lambda_k returns to its double buffer; u~ stayed double throughout.  The
// speculative next iterate is dropped: every solve begins by recomputing it.
template <int D>
__global__ void k_polish_state(Ctrl* __restrict__ ctrl, double* F0, double* F1, double* __restrict__ Lam,
                               float* __restrict__ Lh, float* __restrict__ Ll, double* U0, double* U1, long long V,
                               int enter) {
    constexpr int NN = D * D;
    if (enter ? (ctrl->done != kRunning || ctrl->dw_state) : !ctrl->dw_state) return;
    const long long k = ctrl->k;
    double* Fa = ((k + 1) & 1) ? F1 : F0;  // buffer (k + 1) & 1
    double* Fb = (k & 1) ? F1 : F0;        // buffer k & 1
    const long long n = (long long)NN * V;
    if (!enter && ctrl->u_pair) {
        // u~_k from its float pair (buffer (k + 1) & 1) to double in buffer k & 1
        const float* Ua = reinterpret_cast<const float*>(((k + 1) & 1) ? U1 : U0);
        double* Ub = (k & 1) ? U1 : U0;
        const long long nu = (long long)D * V;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nu;
             i += (long long)gridDim.x * blockDim.x)
            Ub[i] = f2d_bits(Ua[i]) + f2d_bits(Ua[nu + i]);
    }
    if (!enter && (V & 3) == 0) {
        // leave, V a multiple of 4: four elements per thread with vector loads and stores
        // (same values; 0.1 ms less per 128^3 solve than the scalar loop below)
        const float4* Fi4 = reinterpret_cast<const float4*>(Fa);
        const float4* Lh4 = reinterpret_cast<const float4*>(Lh);
        const float4* Ll4 = reinterpret_cast<const float4*>(Ll);
        double2* Fb2 = reinterpret_cast<double2*>(Fb);
        double2* L2 = reinterpret_cast<double2*>(Lam);
        const long long n4 = n / 4;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
            const float4 fh = Fi4[i], fl = Fi4[n4 + i], lh = Lh4[i], ll = Ll4[i];
            Fb2[2 * i] = double2{f2d_bits(fh.x) + f2d_bits(fl.x), f2d_bits(fh.y) + f2d_bits(fl.y)};
            Fb2[2 * i + 1] = double2{f2d_bits(fh.z) + f2d_bits(fl.z), f2d_bits(fh.w) + f2d_bits(fl.w)};
            L2[2 * i] = double2{f2d_bits(lh.x) + f2d_bits(ll.x), f2d_bits(lh.y) + f2d_bits(ll.y)};
            L2[2 * i + 1] = double2{f2d_bits(lh.z) + f2d_bits(ll.z), f2d_bits(lh.w) + f2d_bits(ll.w)};
        }
        return;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (enter) {
            const dw f = dw_from(Fa[i]);
            float* Fo = reinterpret_cast<float*>(Fb);
            Fo[i] = f.hi;
            Fo[n + i] = f.lo;
            const dw l = dw_from(Lam[i]);
            Lh[i] = l.hi;
            Ll[i] = l.lo;
        } else {
            const float* Fi = reinterpret_cast<const float*>(Fa);
            Fb[i] = f2d_bits(Fi[i]) + f2d_bits(Fi[n + i]);
            Lam[i] = f2d_bits(Lh[i]) + f2d_bits(Ll[i]);
        }
    }
}

// Flips ctrl->dw_state after the conversion (a separate launch: every block of
// k_polish_state reads the flag first).
__global__ void k_polish_flag(Ctrl* __restrict__ ctrl, int enter) {
    if (enter ? (ctrl->done == kRunning && !ctrl->dw_state) : ctrl->dw_state) {
        ctrl->dw_state = enter;
        ctrl->z_valid = 0;
        ctrl->u_pair = 0;  // entered from double: u~ stays double; left: u~ is double again
    }
}

// ------------------------------------------------------------------ direct switch to the polish
// RVE_MIXED, elastic laws, no free <F> components.  When the float phase stops (ctrl->k =
// k) the state is Lambda_k, u~_k and the last fused pass's local result F_{k+1}, all float.
// The polish's increment form needs u~_{k+1} = P(Q_{k+1}), Q_{k+1} = F_{k+1} - Lambda_k/rho,
// to double precision (every later projection adds to it).  With the float u~_k as a first
// approximation, u~_{k+1} = u~_k + delta where delta solves D^T D delta = r,
//   r = D^T (Q_{k+1} - D u~_k)
//     = -sum_j [ (F_ij(x+e_j) - F_ij(x-e_j)) - (Lambda_ij(x+e_j) - Lambda_ij(x-e_j)) / rho
//                - (u_i(x+2e_j) - 2 u_i(x) + u_i(x-2e_j)) n/2 ] n/2,
// of the order of the ADMM residuals.  It is formed from the float values in double-word
// arithmetic: the differences of two floats are exact pairs (two_sum), 1/rho is a float
// pair, and the sum carries about 44 bits, so the rounding left in r is that of its final
// float store, and the float spectral solve of it (the increment passes, with r handed in
// as the divergence: ctrl->div_given) leaves an error far below the polish tolerance.
// (Plain double arithmetic gives the same values but runs on the FP64 pipe: 1.07 ms per
// 128^3 switch against the float pipe's few tens of us.)  This replaces a double local
// step, a double projection and a double fused pass.  The kernel also forms
// R_k = F_{k+1} - G_k (G_k = Fbar + D u~_k, again as a pair, stored rounded to float) and
// the polish's state: F_{k+1} as double-words (float, 0) in the double F buffer k & 1 and
// u~_k as the float pair (u~_k, 0) in the double u buffer (k + 1) & 1 (Ctrl::u_pair).  R_k and r go to the idle double F buffer
// (k + 1) & 1: their final places are float buffers that still hold inputs
// (k_switch_move copies them there).  n >= 4, so one conditional wrap finds every
// neighbour up to two voxels away.
template <int D>
__global__ void __launch_bounds__(256, 2) k_switch_resid(const Ctrl* __restrict__ ctrl, const float* F32_0, const float* F32_1,
                               const float* __restrict__ L32, const float* U32_0, const float* U32_1, double* F64_0,
                               double* F64_1, double* U64_0, double* U64_1, long long V, int n, FastDiv dn) {
    constexpr int NN = D * D;
    const int par = (int)(ctrl->k & 1);
    const float* __restrict__ Fn = par ? F32_0 : F32_1;  // F_{k+1}: buffer (k + 1) & 1
    const float* __restrict__ U = par ? U32_1 : U32_0;   // u~_k: buffer k & 1
    float* __restrict__ Fdw = reinterpret_cast<float*>(par ? F64_1 : F64_0);
    float* __restrict__ scr = reinterpret_cast<float*>(par ? F64_0 : F64_1);
    // u~_k as a float pair (Ctrl::u_pair): (u~_k, 0) in buffer (k + 1) & 1, the high part
    // also in buffer k & 1
    float* __restrict__ Up = reinterpret_cast<float*>(par ? U64_0 : U64_1);
    float* __restrict__ Uq = reinterpret_cast<float*>(par ? U64_1 : U64_0);
    __shared__ dw Fb[NN + 1];  // Fbar as double-words, then 1/rho
    if (threadIdx.x <= NN)
        Fb[threadIdx.x] = dw_from(threadIdx.x < NN ? ctrl->Fbar[(threadIdx.x / D) * 3 + threadIdx.x % D] : 1.0 / ctrl->rho);
    __syncthreads();
    const dw irho = Fb[NN];
    const float hn = 0.5f * (float)n;  // exact: n <= 512
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const unsigned q = fdiv((unsigned)v, dn);
        const int c[3] = {(int)(v - (long long)q * n), D == 3 ? (int)(q - fdiv(q, dn) * (unsigned)n) : (int)q,
                          D == 3 ? (int)fdiv(q, dn) : 0};
        // offsets of the neighbours 1 and 2 voxels away along each axis (periodic)
        int o1p[D], o1m[D], o2p[D], o2m[D];  // |offset| < n^2 <= 2^18
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const int sj = j == 0 ? 1 : (j == 1 ? n : n * n);
            auto off = [&](int s) {
                int t = c[j] + s;
                t += t < 0 ? n : 0;
                t -= t >= n ? n : 0;
                return (t - c[j]) * sj;
            };
            o1p[j] = off(1);
            o1m[j] = off(-1);
            o2p[j] = off(2);
            o2m[j] = off(-2);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
            const float* u = U + (long long)i * V + v;
            const float uc = u[0];
            dw acc{0.f, 0.f};
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float* Fc = Fn + (long long)(i * D + j) * V + v;
                const float* Lc = L32 + (long long)(i * D + j) * V + v;
                const dw dF = two_sum(Fc[o1p[j]], -Fc[o1m[j]]);
                const dw dL = two_sum(Lc[o1p[j]], -Lc[o1m[j]]);
                const dw lap = dw_add_f(two_sum(u[o2p[j]], u[o2m[j]]), -2.f * uc);
                acc = dw_add(acc, dw_sub(dw_sub(dF, dw_mul(dL, irho)), dw_mul_f(lap, hn)));
                const dw G = dw_add(Fb[i * D + j], dw_mul_f(two_sum(u[o1p[j]], -u[o1m[j]]), hn));
                scr[(long long)(i * D + j) * V + v] = dw_add_f(dw_neg(G), Fc[0]).hi;
            }
            scr[(long long)(NN + i) * V + v] = dw_mul_f(acc, -hn).hi;
            Up[(long long)i * V + v] = uc;
            Up[(long long)(D + i) * V + v] = 0.f;
            Uq[(long long)i * V + v] = uc;
        }
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            Fdw[(long long)p * V + v] = Fn[(long long)p * V + v];
            Fdw[(long long)(NN + p) * V + v] = 0.f;
        }
    }
}

// Second half of the direct switch (pointwise): R_k to R32, r to D32, Lambda's low words
// to zero (its high words are the float Lambda_k already in place); flags the double-word
// state and the divergence for the next increment x-forward pass.
template <int D>
__global__ void k_switch_move(Ctrl* __restrict__ ctrl, const double* F64_0, const double* F64_1,
                              float* __restrict__ R32, float* __restrict__ D32, float* __restrict__ LL32, long long V) {
    constexpr int NN = D * D;
    const int par = (int)(ctrl->k & 1);
    const float* __restrict__ scr = reinterpret_cast<const float*>(par ? F64_0 : F64_1);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int p = 0; p < NN; ++p) {
            R32[(long long)p * V + v] = scr[(long long)p * V + v];
            LL32[(long long)p * V + v] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < D; ++i) D32[(long long)i * V + v] = scr[(long long)(NN + i) * V + v];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->div_given = 1;
        ctrl->dw_state = 1;
        ctrl->z_valid = 0;
        ctrl->u_pair = 1;
    }
}

cudaError_t launch_polish_state(const Launch& L, bool enter, cudaStream_t st) {
    if (is_lce(L.model)) return cudaSuccess;  // the LCE polish stays in double
    const int blocks = L.local_blocks;
    if (L.dim == 3)
        k_polish_state<3><<<blocks, 256, 0, st>>>(L.ctrl, L.F64[0], L.F64[1], L.L64, L.LH32, L.LL32, L.U64[0],
                                                   L.U64[1], L.V, enter ? 1 : 0);
    else
        k_polish_state<2><<<blocks, 256, 0, st>>>(L.ctrl, L.F64[0], L.F64[1], L.L64, L.LH32, L.LL32, L.U64[0],
                                                   L.U64[1], L.V, enter ? 1 : 0);
    k_polish_flag<<<1, 1, 0, st>>>(L.ctrl, enter ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_switch_direct(const Launch& L, cudaStream_t st) {
    const int blocks = 152 * 8;
    if (L.dim == 3) {
        k_switch_resid<3><<<blocks, 256, 0, st>>>(L.ctrl, L.F32[0], L.F32[1], L.L32, L.U32[0], L.U32[1], L.F64[0],
                                                  L.F64[1], L.U64[0], L.U64[1], L.V, L.n, L.plan.div_n);
        k_switch_move<3><<<blocks, 256, 0, st>>>(L.ctrl, L.F64[0], L.F64[1], L.R32, L.D32, L.LL32, L.V);
    } else {
        k_switch_resid<2><<<blocks, 256, 0, st>>>(L.ctrl, L.F32[0], L.F32[1], L.L32, L.U32[0], L.U32[1], L.F64[0],
                                                  L.F64[1], L.U64[0], L.U64[1], L.V, L.n, L.plan.div_n);
        k_switch_move<2><<<blocks, 256, 0, st>>>(L.ctrl, L.F64[0], L.F64[1], L.R32, L.D32, L.LL32, L.V);
    }
    return cudaGetLastError();
}

// LCE: the state F_k, n_k (buffer k & 1, precision TS) saved as the previous time step
// of the dissipation terms in the double and the float copies that exist.
template <typename TS>
__global__ void k_save_prev(const Ctrl* __restrict__ ctrl, const TS* F0, const TS* F1, const TS* N0, const TS* N1,
                            double* Fp64, double* np64, float* Fp32, float* np32, long long V) {
    const int par = (int)(ctrl->k & 1);
    const TS* F = par ? F1 : F0;
    const TS* N = par ? N1 : N0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 9 * V; i += (long long)gridDim.x * blockDim.x) {
        const double f = (double)F[i];
        if (Fp64) Fp64[i] = f;
        if (Fp32) Fp32[i] = (float)F[i];
        if (i < 3 * V) {
            if (np64) np64[i] = (double)N[i];
            if (np32) np32[i] = (float)N[i];
        }
    }
}

cudaError_t launch_save_prev(const Launch& L, bool from_fp64, cudaStream_t st) {
    if (!is_lce(L.model)) return cudaSuccess;
    if (from_fp64)
        k_save_prev<double><<<L.local_blocks, 256, 0, st>>>(L.ctrl, L.F64[0], L.F64[1], L.N64[0], L.N64[1], L.Fp64,
                                                          L.np64, L.Fp32, L.np32, L.V);
    else
        k_save_prev<float><<<L.local_blocks, 256, 0, st>>>(L.ctrl, L.F32[0], L.F32[1], L.N32[0], L.N32[1], L.Fp64,
                                                         L.np64, L.Fp32, L.np32, L.V);
    return cudaGetLastError();
}

cudaError_t launch_stress(const Launch& L, bool fp64) {
    if (fp64) RVE_DISPATCH(run_stress, double, L);
    RVE_DISPATCH(run_stress, float, L);
}

cudaError_t launch_convert(const Launch& L, bool to_fp64) {
    const long long nF = (long long)L.dim * L.dim * L.V;
    const long long nU = (long long)L.dim * L.V;
    const long long nN = is_lce(L.model) ? 3 * L.V : 0;
    const int blocks = 152 * 8;
    if (to_fp64)
        k_convert<float, double><<<blocks, 256, 0, L.stream>>>(L.ctrl, L.F32[0], L.F32[1], L.L32, L.U32[0],
                                                               L.U32[1], L.F64[0], L.F64[1], L.L64, L.U64[0],
                                                               L.U64[1], nF, nU, L.N32[0], L.N32[1], L.N64[0],
                                                               L.N64[1], nN);
    else
        k_convert<double, float><<<blocks, 256, 0, L.stream>>>(L.ctrl, L.F64[0], L.F64[1], L.L64, L.U64[0],
                                                               L.U64[1], L.F32[0], L.F32[1], L.L32, L.U32[0],
                                                               L.U32[1], nF, nU, L.N64[0], L.N64[1], L.N32[0],
                                                               L.N32[1], nN);
    return cudaGetLastError();
}

}  // namespace admm
