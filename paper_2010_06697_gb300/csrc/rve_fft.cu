// Spectral Helmholtz projection, Zhou & Bhattacharya Section 2.1 Step 2 (eq. helm)
// solved in Fourier space (eq. helmf) on the periodic cell of Section 2.3:
//
//   D^T D u~_{i+1} = D^T (F_{i+1} - Lambda_i / rho),
//
// D the central-difference gradient (symbol i k_j, k_j = sin(h xi_j)/h), so the
// Laplacian symbol is |k|^2 = sum_j k_j^2 and u^ = (D^T Q)^ / |k|^2, u^ = 0 where
// |k|^2 = 0.  The divergence D^T Q is taken in real space inside the first FFT
// pass; per component the rest is a scalar periodic Poisson solve.
//
// Pass structure per iteration (3D; 2D drops the y pass pair):
//   k_xfwd   divergence stencil of Q = F - Lambda/rho, real-to-complex FFT along x
//   k_faxis  forward FFT along y
//   k_faxis  forward FFT along z, multiply by 2/(N^d |k|^2), inverse FFT along z
//   k_faxis  inverse FFT along y
//   k_xinv   complex-to-real inverse FFT along x -> u~_{i+1}
// The spectrum of u~_{i+1} is built in the buffer that held u~_{i-1} (dead once
// the fused local kernel of iteration i has run), so no extra field is stored.
//
// Real-to-complex along x: a real line of N points is read as N/2 complex
// points z_m = r_{2m} + i r_{2m+1}, transformed at length N/2 and split into the
// N/2+1 bins of the real transform.  Bins 0 and N/2 are real and their symbol
// k_x vanishes at both, so they are stored together as one complex value
// (X_0 + i X_{N/2}); every x-line then holds exactly N/2 complex bins and the
// spectrum occupies the same bytes as the real field.
//
// Each 1D transform is a self-sorting Stockham FFT (radix 8/4/3/2) staged in
// shared memory; x-lines are read and written as contiguous rows, y/z lines as
// tiles of TK adjacent columns so that every global access is a coalesced row
// segment.  Twiddles come from a per-grid table exp(-2 pi i m / N) computed on
// the host in double.
#include <stdint.h>

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "rve_internal.cuh"

namespace admm {
namespace {

template <typename T>
struct Cx;
template <>
struct Cx<double> { using t = double2; };
template <>
struct Cx<float> { using t = float2; };

template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) { return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename V>
__device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
template <typename V>
__device__ __forceinline__ V mul_i(V a) { return V{-a.y, a.x}; }   // i a
template <typename V>
__device__ __forceinline__ V mul_mi(V a) { return V{a.y, -a.x}; }  // -i a
template <typename V, typename S>
__device__ __forceinline__ V cscale(V a, S s) { return V{a.x * s, a.y * s}; }

// Small DFTs, sign -1 (forward) or +1 (INV), unnormalised.
template <bool INV, typename V>
__device__ __forceinline__ void dft2(V* v) {
    const V a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}
template <bool INV, typename V>
__device__ __forceinline__ void dft3(V* v) {
    using S = decltype(v[0].x);
    const S c = S(0.86602540378443864676);  // sin(2 pi / 3)
    const V s12 = cadd(v[1], v[2]);
    const V d12 = cscale(csub(v[1], v[2]), c);
    const V t = csub(v[0], cscale(s12, S(0.5)));
    v[0] = cadd(v[0], s12);
    const V jd = INV ? mul_i(d12) : mul_mi(d12);
    v[1] = cadd(t, jd);
    v[2] = csub(t, jd);
}
template <bool INV, typename V>
__device__ __forceinline__ void dft4(V& a0, V& a1, V& a2, V& a3) {
    const V s02 = cadd(a0, a2), d02 = csub(a0, a2);
    const V s13 = cadd(a1, a3), d13 = csub(a1, a3);
    const V jd = INV ? mul_i(d13) : mul_mi(d13);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, jd);
    a3 = csub(d02, jd);
}
template <bool INV, typename V>
__device__ __forceinline__ void dft4(V* v) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
}
template <bool INV, typename V>
__device__ __forceinline__ void dft8(V* v) {
    using S = decltype(v[0].x);
    const S r = S(0.70710678118654752440);  // 1/sqrt(2)
    V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    V o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    // twiddles W8^1, W8^2, W8^3 with W8 = exp(-+ i pi/4)
    if (INV) {
        o1 = V{(o1.x - o1.y) * r, (o1.x + o1.y) * r};
        o2 = mul_i(o2);
        o3 = V{(-o3.x - o3.y) * r, (o3.x - o3.y) * r};
    } else {
        o1 = V{(o1.x + o1.y) * r, (o1.y - o1.x) * r};
        o2 = mul_mi(o2);
        o3 = V{(o3.y - o3.x) * r, -(o3.x + o3.y) * r};
    }
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <int R, bool INV, typename V>
__device__ __forceinline__ void dft(V* v) {
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 3) dft3<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v);
    else dft8<INV>(v);
}

// One Stockham pass of radix R over `nl` independent transforms of length L
// held in shared memory.  Element e of transform l sits at l*ls + e*es.  P holds
// nb = L/R, Ns (the product of the radices already applied) and the twiddle
// stride.  Output is in natural order after the last pass.  COLS: consecutive
// threads take consecutive transforms (tiles of columns); otherwise consecutive
// butterflies of one transform.
template <int R, bool INV, bool COLS, typename V>
__device__ __forceinline__ void stockham_pass(const V* __restrict__ src, V* __restrict__ dst,
                                              const V* __restrict__ tw, const FftPass& P, const FastDiv& nl,
                                              int ls, int es) {
    const unsigned nb = P.nb.d, Ns = P.ns.d;
    const unsigned total = nb * nl.d;
    const int tstep = P.tstep;
    for (unsigned t = threadIdx.x; t < total; t += blockDim.x) {
        unsigned l, j;
        if (COLS) {
            j = fdiv(t, nl);
            l = t - j * nl.d;
        } else {
            l = fdiv(t, P.nb);
            j = t - l * nb;
        }
        const int base = (int)l * ls;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[base + (int)(j + r * nb) * es];
        const unsigned kk = j - fdiv(j, P.ns) * Ns;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                V w = tw[r * (int)kk * tstep];
                if (INV) w = cconj(w);
                v[r] = cmul(v[r], w);
            }
        }
        dft<R, INV>(v);
        const int d0 = (int)((j - kk) * R + kk);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + (d0 + r * (int)Ns) * es] = v[r];
    }
}

// All passes of one transform; returns the buffer holding the result.
template <bool INV, bool COLS, typename V>
__device__ V* stockham(V* a, V* b, const V* tw, const int* rad, const FftPass* passes, int np, const FastDiv& nl,
                       int ls, int es) {
    V* src = a;
    V* dst = b;
    for (int p = 0; p < np; ++p) {
        const FftPass& P = passes[p];
        switch (rad[p]) {
            case 2: stockham_pass<2, INV, COLS>(src, dst, tw, P, nl, ls, es); break;
            case 3: stockham_pass<3, INV, COLS>(src, dst, tw, P, nl, ls, es); break;
            case 4: stockham_pass<4, INV, COLS>(src, dst, tw, P, nl, ls, es); break;
            default: stockham_pass<8, INV, COLS>(src, dst, tw, P, nl, ls, es); break;
        }
        __syncthreads();
        V* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

template <typename V>
__device__ __forceinline__ void load_twiddles(V* s_tw, const V* __restrict__ g_tw, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_tw[i] = g_tw[i];
}

template <typename T>
struct FftArgs;
template <>
struct FftArgs<double> {
    __host__ __device__ static double* U(const Launch& L, int i) { return L.U64[i]; }
    __host__ __device__ static const double* F(const Launch& L, int i) { return L.F64[i]; }
    __host__ __device__ static const double* Lm(const Launch& L) { return L.L64; }
    __host__ __device__ static const double2* tw(const Launch& L) { return L.tw64; }
    __host__ __device__ static const double* ksq(const Launch& L) { return L.ksq64; }
    __host__ __device__ static int tile(const Launch& L) { return L.tk64; }
    __host__ __device__ static double half_n(const Launch& L) { return L.half_n64; }
    __host__ __device__ static double scale(const Launch& L) { return L.scale64; }
    __host__ __device__ static const FastDiv& tile_div(const Launch& L) { return L.plan.div_tk64; }
    static constexpr int tk = 8;
};
template <>
struct FftArgs<float> {
    __host__ __device__ static float* U(const Launch& L, int i) { return L.U32[i]; }
    __host__ __device__ static const float* F(const Launch& L, int i) { return L.F32[i]; }
    __host__ __device__ static const float* Lm(const Launch& L) { return L.L32; }
    __host__ __device__ static const float2* tw(const Launch& L) { return L.tw32; }
    __host__ __device__ static const float* ksq(const Launch& L) { return L.ksq32; }
    __host__ __device__ static int tile(const Launch& L) { return L.tk32; }
    __host__ __device__ static float half_n(const Launch& L) { return L.half_n32; }
    __host__ __device__ static float scale(const Launch& L) { return L.scale32; }
    __host__ __device__ static const FastDiv& tile_div(const Launch& L) { return L.plan.div_tk32; }
    static constexpr int tk = 16;
};

// ------------------------------------------------------------------ x passes

// Divergence of Q = F_{k+1} - Lambda_k / rho (D^T Q = minus the central
// divergence) and real-to-complex FFT along x, for `lpb` consecutive x-lines.
// INCR: Q is the increment R given in F0 (= F1), Lambda is not read, and the
// spectrum goes to U0 (= U1).
template <typename T, int D, bool INCR>
__device__ __forceinline__ void xfwd_tile(const Launch& L, int bid, const void*& twp) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    const T* F0 = INCR ? (const T*)L.R32 : Args::F(L, 0);
    const T* F1 = INCR ? (const T*)L.R32 : Args::F(L, 1);
    const T* __restrict__ Lam = Args::Lm(L);
    T* U0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* U1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    const V* __restrict__ g_tw = Args::tw(L);
    const FftPlan& plan = L.plan;
    const int lpb = L.lpb;
    if (ctrl->done) return;
    const int n = plan.n, H = n / 2;
    const long long Vn = (D == 3) ? (long long)n * n * n : (long long)n * n;
    const int nlines = (D == 3) ? n * n : n;
    const int par = (int)(ctrl->k & 1);
    const T* __restrict__ F = par ? F0 : F1;  // F_{k+1}
    V* __restrict__ S = reinterpret_cast<V*>(par ? U0 : U1);
    const T inv_rho = (T)ctrl->inv_rho;
    const T half_n = Args::half_n(L);

    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* A = s_tw + n;
    V* B = A + lpb * H;
    T* Ar = reinterpret_cast<T*>(A);
    if (twp != (const void*)g_tw) {  // the RVE's table, loaded when the block's RVE changes
        load_twiddles(s_tw, g_tw, n);
        twp = g_tw;
    }
    const int line0 = bid * lpb;
    if (line0 >= nlines) return;  // tiles counted for the fixed kernels' one component each
    const FastDiv nl{(unsigned)lpb, 0u, 0u};  // transforms per block (only the count is used)
    const long long sn = n, s2 = sn * sn;

    for (int c = 0; c < D; ++c) {
        const T* F_c0 = F + (long long)(c * D + 0) * Vn;
        const T* F_c1 = F + (long long)(c * D + 1) * Vn;
        const T* L_c0 = INCR ? nullptr : Lam + (long long)(c * D + 0) * Vn;
        const T* L_c1 = INCR ? nullptr : Lam + (long long)(c * D + 1) * Vn;
        bool vectorised = false;
        if (INCR && ctrl->div_given) {  // the switch to the polish handed in D^T W itself (D32)
            vectorised = true;
            const T* Dg = (const T*)L.D32 + (long long)c * Vn;
            for (int idx = threadIdx.x; idx < lpb * n; idx += blockDim.x) {
                const int l = (int)fdiv(idx, plan.div_n);
                const int line = line0 + l;
                Ar[idx] = line < nlines ? Dg[(long long)line * n + (idx - l * n)] : T(0);
            }
        } else if constexpr (std::is_same<T, float>::value) {
            if ((n & 3) == 0) {
                vectorised = true;
                // four consecutive x per thread (n a multiple of 4): float4 loads of the
                // centre row and of the y and z neighbour rows (fields 256-byte aligned); the
                // x neighbours of the end elements come from the adjacent lanes, or from memory
                // at a line's ends (periodic wrap) and at a warp's ends.  Every lane of a warp
                // runs every pass of the loop, so the shuffles see full warps.  The same
                // arithmetic per element, in the same order, as the scalar form below.
                const int lane = threadIdx.x & 31;
                const int total = lpb * n / 4;
                for (int base = 0; base < total; base += blockDim.x) {
                    const int qd = base + threadIdx.x;
                    const int e = 4 * qd;
                    const int l = (int)fdiv(e, plan.div_n);
                    const int x = e - l * n;
                    const int line = line0 + l;
                    const bool act = qd < total && line < nlines;
                    const long long v = (long long)line * n + x;
                    long long yp = v, ym = v, zp = v, zm = v;
                    if (act) {
                        const int zq = (int)fdiv(line, plan.div_n);
                        const int y = line - zq * n;
                        yp = v + (y + 1 == n ? (1 - n) * sn : sn);
                        ym = v + (y == 0 ? (n - 1) * sn : -sn);
                        if constexpr (D == 3) {
                            zp = v + (zq + 1 == n ? (1 - n) * s2 : s2);
                            zm = v + (zq == 0 ? (n - 1) * s2 : -s2);
                        }
                    }
                    // all loads of the element group issued before the first use (as in
                    // xfwd_fixed_tile), the line- and warp-end x neighbours among them
                    auto ld4 = [](const float* p) { return *reinterpret_cast<const float4*>(p); };
                    const float* A0[2] = {F_c0, L_c0};
                    const float* A1[2] = {F_c1, L_c1};
                    const float* A2[2] = {F + (long long)(c * D + 2) * Vn,
                                          INCR ? nullptr : Lam + (long long)(c * D + 2) * Vn};
                    constexpr int NA = INCR ? 1 : 2;
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const bool wl = act && (x == 0 || lane == 0), wr = act && (x + 4 == n || lane == 31);
                    float4 ac[2], ap[2], am[2], au[2] = {z4, z4}, ad[2] = {z4, z4};
                    float el[2] = {}, er[2] = {};
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        ac[a] = act ? ld4(A0[a] + v) : z4;
                        ap[a] = act ? ld4(A1[a] + yp) : z4;
                        am[a] = act ? ld4(A1[a] + ym) : z4;
                        if constexpr (D == 3) {
                            if (act) {
                                au[a] = ld4(A2[a] + zp);
                                ad[a] = ld4(A2[a] + zm);
                            }
                        }
                        if (wl) el[a] = A0[a][v + (x == 0 ? n - 1 : -1)];
                        if (wr) er[a] = A0[a][v + (x + 4 == n ? 4 - n : 4)];
                    }
                    float dx[2][4], dy[2][4] = {}, dz[2][4] = {};
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        const float4 ctr = ac[a];
                        float left = __shfl_sync(0xffffffffu, ctr.w, (lane + 31) & 31);
                        float right = __shfl_sync(0xffffffffu, ctr.x, (lane + 1) & 31);
                        if (wl) left = el[a];
                        if (wr) right = er[a];
                        if (act) {
                            dy[a][0] = ap[a].x - am[a].x;
                            dy[a][1] = ap[a].y - am[a].y;
                            dy[a][2] = ap[a].z - am[a].z;
                            dy[a][3] = ap[a].w - am[a].w;
                            if constexpr (D == 3) {
                                dz[a][0] = au[a].x - ad[a].x;
                                dz[a][1] = au[a].y - ad[a].y;
                                dz[a][2] = au[a].z - ad[a].z;
                                dz[a][3] = au[a].w - ad[a].w;
                            }
                        }
                        dx[a][0] = ctr.y - left;
                        dx[a][1] = ctr.z - ctr.x;
                        dx[a][2] = ctr.w - ctr.y;
                        dx[a][3] = right - ctr.z;
                    }
                    const float* fx = dx[0];
                    const float* fy = dy[0];
                    const float* fz = dz[0];
                    const float* lx = dx[1];
                    const float* ly = dy[1];
                    const float* lz = dz[1];
                    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (act) {
                        float r[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            T q = fx[k] + fy[k];
                            if (!INCR) q -= (lx[k] + ly[k]) * inv_rho;
                            if constexpr (D == 3) {
                                q += fz[k];
                                if (!INCR) q -= lz[k] * inv_rho;
                            }
                            r[k] = -q * half_n;
                        }
                        o = make_float4(r[0], r[1], r[2], r[3]);
                    }
                    if (qd < total) *reinterpret_cast<float4*>(Ar + e) = o;
                }
            }
        }
        for (int idx = threadIdx.x; !vectorised && idx < lpb * n; idx += blockDim.x) {
            const int l = (int)fdiv(idx, plan.div_n);
            const int x = idx - l * n;
            const int line = line0 + l;
            T r = T(0);
            if (line < nlines) {
                const int zq = (int)fdiv(line, plan.div_n);
                const int y = line - zq * n;
                const long long v = (long long)line * n + x;
                const long long xp = v + (x + 1 == n ? 1 - n : 1), xm = v + (x == 0 ? n - 1 : -1);
                const long long yp = v + (y + 1 == n ? (1 - n) * sn : sn), ym = v + (y == 0 ? (n - 1) * sn : -sn);
                T q = (F_c0[xp] - F_c0[xm]) + (F_c1[yp] - F_c1[ym]);
                if (!INCR) q -= ((L_c0[xp] - L_c0[xm]) + (L_c1[yp] - L_c1[ym])) * inv_rho;
                if constexpr (D == 3) {
                    const int z = zq;
                    const T* F_c2 = F + (long long)(c * D + 2) * Vn;
                    const long long zp = v + (z + 1 == n ? (1 - n) * s2 : s2);
                    const long long zm = v + (z == 0 ? (n - 1) * s2 : -s2);
                    q += F_c2[zp] - F_c2[zm];
                    if (!INCR) {
                        const T* L_c2 = Lam + (long long)(c * D + 2) * Vn;
                        q -= (L_c2[zp] - L_c2[zm]) * inv_rho;
                    }
                }
                r = -q * half_n;
            }
            Ar[idx] = r;
        }
        __syncthreads();
        V* X = stockham<false, false>(A, B, s_tw, plan.rad_half, plan.pass_half, plan.np_half, nl, H, 1);
        V* S_c = S + (long long)c * (Vn / 2);
        for (int idx = threadIdx.x; idx < lpb * H; idx += blockDim.x) {
            const int l = (int)fdiv(idx, plan.div_h);
            const int kk = idx - l * H;
            const int line = line0 + l;
            if (line >= nlines) continue;
            const V Zk = X[l * H + kk];
            V out;
            if (kk == 0) {
                out = V{Zk.x + Zk.y, Zk.x - Zk.y};  // (X_0, X_{N/2}) packed
            } else {
                const V Zc = cconj(X[l * H + (H - kk)]);
                const V E = cscale(cadd(Zk, Zc), T(0.5));
                const V O = cscale(mul_mi(csub(Zk, Zc)), T(0.5));
                out = cadd(E, cmul(s_tw[kk], O));
            }
            S_c[(long long)line * H + kk] = out;
        }
        __syncthreads();
    }
}

// Complex-to-real inverse FFT along x.  Plain: in place, spectrum lines in the
// buffer of u~_{k+1} (S0/S1 by parity) become u~_{k+1} (TO = T, O = S).
// INCR: the spectrum of P(R) sits in S0; u~_{k+1} = u~_k + P(R) is written in
// the precision TO of the state buffers O0/O1.
// INCR also stores the float increment itself in DUout (read by the next local step for r_d).
template <typename T, typename TO, int D, bool INCR>
__device__ __forceinline__ void xinv_tile(const Launch& L, int bid, const void*& twp) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    T* S0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* S1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    TO* O0 = INCR ? (TO*)L.U64[0] : (TO*)Args::U(L, 0);
    TO* O1 = INCR ? (TO*)L.U64[1] : (TO*)Args::U(L, 1);
    T* __restrict__ DUout = (T*)L.D32;
    const V* __restrict__ g_tw = Args::tw(L);
    const FftPlan& plan = L.plan;
    const int lpb = L.lpb;
    if (ctrl->done) return;
    const int n = plan.n, H = n / 2;
    const long long Vn = (D == 3) ? (long long)n * n * n : (long long)n * n;
    const int nlines = (D == 3) ? n * n : n;
    const int par = (int)(ctrl->k & 1);
    V* S = reinterpret_cast<V*>(INCR ? S0 : (par ? S0 : S1));
    // u~ as float pairs (Ctrl::u_pair): the low parts of u~_k (pair buffer (k + 1) & 1) and
    // of u~_{k+1} (buffer k & 1); the high parts stay as written at the switch
    const bool upair = INCR && ctrl->u_pair;
    const float* Plo_in = INCR ? reinterpret_cast<const float*>(par ? L.U64[0] : L.U64[1]) + D * Vn : nullptr;
    float* Plo_out = INCR ? reinterpret_cast<float*>(par ? L.U64[1] : L.U64[0]) + D * Vn : nullptr;
    TO* Out = par ? O0 : O1;
    const TO* In = par ? O1 : O0;
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* A = s_tw + n;
    V* B = A + lpb * H;
    if (twp != (const void*)g_tw) {  // the RVE's table, loaded when the block's RVE changes
        load_twiddles(s_tw, g_tw, n);
        twp = g_tw;
    }
    __syncthreads();
    const int line0 = bid * lpb;
    if (line0 >= nlines) return;  // tiles counted for the fixed kernels' one component each
    const FastDiv nl{(unsigned)lpb, 0u, 0u};  // transforms per block (only the count is used)
    for (int c = 0; c < D; ++c) {
        V* S_c = S + (long long)c * (Vn / 2);
        for (int idx = threadIdx.x; idx < lpb * H; idx += blockDim.x) {
            const int l = (int)fdiv(idx, plan.div_h);
            const int kk = idx - l * H;
            const int line = line0 + l;
            V Z = V{T(0), T(0)};
            if (line < nlines) {
                const V Xk = S_c[(long long)line * H + kk];
                if (kk == 0) {
                    Z = V{T(0.5) * (Xk.x + Xk.y), T(0.5) * (Xk.x - Xk.y)};
                } else {
                    const V Xc = cconj(S_c[(long long)line * H + (H - kk)]);
                    const V E = cscale(cadd(Xk, Xc), T(0.5));
                    const V O = cmul(cscale(csub(Xk, Xc), T(0.5)), cconj(s_tw[kk]));
                    Z = cadd(E, mul_i(O));
                }
            }
            A[idx] = Z;
        }
        __syncthreads();
        V* X = stockham<true, false>(A, B, s_tw, plan.rad_half, plan.pass_half, plan.np_half, nl, H, 1);
        const T* Xr = reinterpret_cast<const T*>(X);
        TO* O_c = Out + (long long)c * Vn;
        const TO* I_c = In + (long long)c * Vn;
        bool vectorised = false;
        if constexpr (std::is_same<T, float>::value && std::is_same<TO, float>::value && !INCR) {
            if ((n & 3) == 0) {  // float4 stores of four consecutive x (lines start on 16 bytes)
                vectorised = true;
                for (int qd = threadIdx.x; qd < lpb * n / 4; qd += blockDim.x) {
                    const int e = 4 * qd;
                    const int l = (int)fdiv(e, plan.div_n);
                    const int line = line0 + l;
                    if (line < nlines)
                        *reinterpret_cast<float4*>(O_c + (long long)line * n + (e - l * n)) =
                            *reinterpret_cast<const float4*>(Xr + e);
                }
            }
        }
        for (int idx = threadIdx.x; !vectorised && idx < lpb * n; idx += blockDim.x) {
            const int l = (int)fdiv(idx, plan.div_n);
            const int line = line0 + l;
            if (line < nlines) {
                const long long o = (long long)line * n + (idx - l * n);
                if (INCR) {
                    if (upair)
                        Plo_out[(long long)c * Vn + o] = Plo_in[(long long)c * Vn + o] + (float)Xr[idx];
                    else
                        O_c[o] = I_c[o] + (TO)Xr[idx];
                    DUout[(long long)c * Vn + o] = Xr[idx];
                } else
                    O_c[o] = (TO)Xr[idx];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ y / z passes

// FFT along AXIS (1 = y, 2 = z) of tiles of `tk` adjacent x-frequency columns.
// MODE 0: forward; 1: inverse; 2: forward, multiply by scale/|k|^2, inverse.
template <typename T, int D, int AXIS, int MODE, bool INCR>
__device__ __forceinline__ void faxis_tile(const Launch& L, int bid, const void*& twp) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    T* U0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* U1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    const V* __restrict__ g_tw = Args::tw(L);
    const T* __restrict__ ksq = Args::ksq(L);
    const FftPlan& plan = L.plan;
    const int tk = Args::tile(L);
    const FastDiv& dtk = Args::tile_div(L);
    const T scale = Args::scale(L);
    if (ctrl->done) return;
    const int n = plan.n, H = n / 2;
    const long long Vn = (D == 3) ? (long long)n * n * n : (long long)n * n;
    const int par = (int)(ctrl->k & 1);
    V* S = reinterpret_cast<V*>(par ? U0 : U1);
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* X = s_tw + n;
    V* Y = X + n * tk;
    if (twp != (const void*)g_tw) {  // the RVE's table, loaded when the block's RVE changes
        load_twiddles(s_tw, g_tw, n);
        twp = g_tw;
    }

    const int gxa = (H + tk - 1) / tk;
    const int gya = (D == 3) ? n : 1;
    const int col0 = (bid % gxa) * tk;
    const int outer = (bid / gxa) % gya;
    const int c = bid / (gxa * gya);
    long long base, es_g;
    if (D == 3 && AXIS == 1) {
        base = (long long)c * (Vn / 2) + (long long)outer * n * H + col0;
        es_g = H;
    } else if (D == 3 && AXIS == 2) {
        base = (long long)c * (Vn / 2) + (long long)outer * H + col0;
        es_g = (long long)n * H;
    } else {
        base = (long long)c * (Vn / 2) + col0;
        es_g = H;
    }
    for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
        const int e = (int)fdiv(idx, dtk);
        const int cl = idx - e * tk;
        X[idx] = (col0 + cl < H) ? S[base + e * es_g + cl] : V{T(0), T(0)};
    }
    __syncthreads();
    V* R;
    if (MODE == 1) {
        R = stockham<true, true>(X, Y, s_tw, plan.rad_full, plan.pass_full, plan.np_full, dtk, 1, tk);
    } else {
        R = stockham<false, true>(X, Y, s_tw, plan.rad_full, plan.pass_full, plan.np_full, dtk, 1, tk);
        if (MODE == 2) {
            const T kout = (D == 3) ? __ldg(ksq + outer) : T(0);
            for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
                const int e = (int)fdiv(idx, dtk);
                const int col = col0 + idx - e * tk;
                const T den = __ldg(ksq + e) + __ldg(ksq + min(col, H - 1)) + kout;
                const T m = den > T(0) ? scale / den : T(0);
                R[idx] = cscale(R[idx], m);
            }
            __syncthreads();
            V* other = (R == X) ? Y : X;
            R = stockham<true, true>(R, other, s_tw, plan.rad_full, plan.pass_full, plan.np_full, dtk, 1, tk);
        }
    }
    for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
        const int e = (int)fdiv(idx, dtk);
        const int cl = idx - e * tk;
        if (col0 + cl < H) S[base + e * es_g + cl] = R[idx];
    }
}

// ------------------------------------------------------------------ fixed-size column passes

// Columns of power-of-two length N in {64, 128, 256, 512}: N/8 threads per column and
// 2048/N columns per block of 256 threads.  Each thread keeps 8 elements of its column
// in registers through all passes (radix 8, then a last radix 2 or 4 where N is not a
// power of 8) and exchanges them through shared memory between passes.  After a whole
// transform a thread holds elements j + (N/8) r again, the positions it loaded, so the
// forward transform, the spectral scaling and the inverse of the z solve follow one
// another in registers.  All index arithmetic is fixed at compile time.
template <int N>
struct ColPlan {
    static constexpr int T = N / 8;                                // threads per column
    static constexpr int TK = 256 / T;                             // columns per block
    static constexpr int P8 = N == 512 ? 3 : 2;                    // radix-8 passes
    static constexpr int RL = N == 128 ? 2 : (N == 256 ? 4 : 1);   // last radix (1: none)
};

// Asynchronous 8-byte global-to-shared copies (cp.async, cached in L1), their commit and
// the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <bool INV, typename V>
__device__ __forceinline__ V twiddled(V a, V w) {
    return cmul(a, INV ? cconj(w) : w);
}

// One Stockham transform (sign by INV, unnormalised) of the block's columns.  x: the
// thread's elements j + T r of column cl, on entry and on exit.  buf: two shared
// buffers of N * S values (element e of column cl at e S + cl; S >= TK, padded for
// the x passes); tw: the table exp(-2 pi i m / (N TWS)) (TWS = 2: the half-length
// transforms of the x passes use every other entry of the grid's table).  ONE: a single
// buffer of N * S values, read and rewritten in place with a barrier in between (the y/z
// passes: half the shared memory, 1 us less per 128^3 pass).
template <int N, bool INV, int TWS = 1, int S = ColPlan<N>::TK, bool ONE = false, typename V>
__device__ __forceinline__ void col_fft(V (&x)[8], V* __restrict__ buf, const V* __restrict__ tw, int j, int cl) {
    using P = ColPlan<N>;
    constexpr int T = P::T, TK = S;
    __syncthreads();  // the previous transform's readers are done with both buffers
#pragma unroll
    for (int p = 0; p < P::P8; ++p) {
        const int Ns = 1 << (3 * p);
        V* in = ONE ? buf : buf + ((p + 1) & 1) * (N * TK);
        V* out = ONE ? buf : buf + (p & 1) * (N * TK);
        const int k = j & (Ns - 1);
        if (p > 0) {
#pragma unroll
            for (int r = 0; r < 8; ++r) x[r] = in[(j + T * r) * TK + cl];
#pragma unroll
            for (int r = 1; r < 8; ++r) x[r] = twiddled<INV>(x[r], tw[k * r * (N / (8 * Ns)) * TWS]);
        }
        dft8<INV>(x);
        const bool last = (p == P::P8 - 1) && P::RL == 1;
        if (!last) {
            if (ONE && p > 0) __syncthreads();  // one buffer: this pass's reads are done
#pragma unroll
            for (int r = 0; r < 8; ++r) out[((j - k) * 8 + r * Ns + k) * TK + cl] = x[r];
            __syncthreads();
        }
    }
    if constexpr (P::RL > 1) {
        constexpr int RL = P::RL, Q = 8 / RL, Ns = N / RL;
        const V* in = ONE ? buf : buf + ((P::P8 - 1) & 1) * (N * TK);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int b = j + T * q;  // butterfly index (< Ns): twiddle exponent b r
            V v[RL];
#pragma unroll
            for (int r = 0; r < RL; ++r) {
                v[r] = in[(b + Ns * r) * TK + cl];
                if (r > 0) v[r] = twiddled<INV>(v[r], tw[b * r * TWS]);
            }
            if constexpr (RL == 2) dft2<INV>(v);
            else dft4<INV>(v);
#pragma unroll
            for (int r = 0; r < RL; ++r) x[q + r * Q] = v[r];  // element b + Ns r = j + T (q + r Q)
        }
    }
}

// xfwd_tile and xinv_tile for 3D grids of N in {128, 256, 512}: the half-length
// transforms (H = N/2) of the block's 4096/N lines run through col_fft with the
// lines as columns; staging, the stencil and the real-to-complex split are those of
// the general kernels (same arithmetic per element; the float instances move four x
// per thread with vector loads and stores), in shared buffers padded to a stride of
// 4096/N + 1 values.
template <int N>
struct XPlan {
    static constexpr int H = N / 2;
    static constexpr int LPB = ColPlan<H>::TK;  // lines per block
    static constexpr int S = LPB + 1;            // padded element stride
    static constexpr int LOGN = N == 128 ? 7 : (N == 256 ? 8 : 9);
};

template <typename T, int N, int D, bool INCR>
__device__ __forceinline__ void xfwd_fixed_tile(const Launch& L, int bid, bool& twl) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    using X = XPlan<N>;
    constexpr int H = X::H, LPB = X::LPB, S = X::S, TT = ColPlan<H>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    const T* F0 = INCR ? (const T*)L.R32 : Args::F(L, 0);
    const T* F1 = INCR ? (const T*)L.R32 : Args::F(L, 1);
    const T* __restrict__ Lam = Args::Lm(L);
    T* U0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* U1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    if (ctrl->done) return;
    constexpr long long Vn = (D == 3) ? (long long)N * N * N : (long long)N * N;
    constexpr int nlines = (D == 3) ? N * N : N;
    const int par = (int)(ctrl->k & 1);
    const T* __restrict__ F = par ? F0 : F1;  // F_{k+1}
    V* __restrict__ Sp = reinterpret_cast<V*>(par ? U0 : U1);
    const T inv_rho = (T)ctrl->inv_rho;
    const T half_n = Args::half_n(L);
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* buf = s_tw + N;          // two buffers of H * S values
    V* stage = buf + H * S;     // the second one stages the input lines
    T* stage_r = reinterpret_cast<T*>(stage);
    if (!twl) {  // exp(-2 pi i m / N) depends on N only: loaded on the block's first tile
        load_twiddles(s_tw, Args::tw(L), N);
        twl = true;
    }
    // one component per tile (tiles_x): three times the blocks of a loop over components,
    // whose load latency then overlaps across blocks instead of adding up within one
    constexpr int NB = nlines / LPB;
    const int c0 = bid / NB;
    const int line0 = (bid % NB) * LPB;
    const int lt = threadIdx.x % LPB, jt = threadIdx.x / LPB;
    // a tile's LPB lines are consecutive y of one z plane (LPB divides N): the z
    // neighbours are fixed offsets.  Voxel indices fit 32 bits (N^3 < 2^31); the
    // increment variant runs faster with them, the plain one (twice the loads) with
    // 64-bit ones (measured on GB300)
    using Idx = typename std::conditional<INCR, int, long long>::type;
    const int z = line0 >> X::LOGN, y0 = line0 & (N - 1);
    constexpr Idx sn = N, s2 = (Idx)N * N;
    const bool divg = INCR && ctrl->div_given;
    const Idx zp = (z + 1 == N ? (1 - N) * s2 : s2), zm = (z == 0 ? (N - 1) * s2 : -s2);
    for (int c = c0; c < c0 + 1; ++c) {
        const T* F_c0 = F + (long long)(c * D + 0) * Vn;
        const T* F_c1 = F + (long long)(c * D + 1) * Vn;
        const T* F_c2 = F + (long long)(c * D + 2) * Vn;
        const T* L_c0 = INCR ? nullptr : Lam + (long long)(c * D + 0) * Vn;
        const T* L_c1 = INCR ? nullptr : Lam + (long long)(c * D + 1) * Vn;
        const T* L_c2 = INCR ? nullptr : Lam + (long long)(c * D + 2) * Vn;
        __syncthreads();  // the previous component's readers of the staging buffer are done
        if constexpr (std::is_same<T, float>::value) {
            // four consecutive x per thread: float4 loads of the centre row and of the y and
            // z neighbour rows (fields are 256-byte aligned, x and N multiples of 4); the x
            // neighbours of the end elements come from the adjacent lanes.  A warp spans 128
            // consecutive x of one line (LPB * N / 4 is a multiple of the block size, so
            // every warp runs every iteration): for N = 128 the lane rotation is the periodic
            // wrap, for longer lines the two warp-end lanes load theirs.  Same arithmetic per
            // element, in the same order, as the scalar form below.
            const int lane = threadIdx.x & 31;
            for (int idx = threadIdx.x; idx < LPB * N / 4; idx += blockDim.x) {
                const int e = idx * 4;
                const int l = e >> X::LOGN;
                const int x = e & (N - 1);
                const int y = y0 + l;
                const Idx v = (Idx)line0 * N + e;
                const Idx yp = v + (y + 1 == N ? (1 - N) * sn : sn), ym = v + (y == 0 ? (N - 1) * sn : -sn);
                // all ten (increment: five) loads of the four elements are issued before the
                // first use: with the loads of the F and the Lambda stencils interleaved
                // with the lane shuffles, the pass took 48.6 us at 128^3 instead of 41.9
                auto ld4 = [](const T* a) { return *reinterpret_cast<const float4*>(a); };
                T o[4];
                if (INCR && divg) {  // the switch to the polish handed in D^T W itself (D32)
                    const float4 g = ld4((const T*)L.D32 + (long long)c * Vn + v);
                    o[0] = g.x;
                    o[1] = g.y;
                    o[2] = g.z;
                    o[3] = g.w;
                } else {
                    float4 ac[2], ap[2], am[2], au[2], ad[2];
                    T el[2] = {}, er[2] = {};  // warp-end x neighbours (N > 128)
                    const T* A0[2] = {F_c0, L_c0};
                    const T* A1[2] = {F_c1, L_c1};
                    const T* A2[2] = {F_c2, L_c2};
                    constexpr int NA = INCR ? 1 : 2;
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        ac[a] = ld4(A0[a] + v);
                        ap[a] = ld4(A1[a] + yp);
                        am[a] = ld4(A1[a] + ym);
                        au[a] = ld4(A2[a] + v + zp);
                        ad[a] = ld4(A2[a] + v + zm);
                        if constexpr (N > 128) {
                            if (lane == 0) el[a] = A0[a][v + (x == 0 ? N - 1 : -1)];
                            if (lane == 31) er[a] = A0[a][v + (x + 4 == N ? 4 - N : 4)];
                        }
                    }
                    T dx[2][4], dy[2][4], dz[2][4];
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        const float4 c = ac[a];
                        T left = __shfl_sync(0xffffffffu, c.w, (lane + 31) & 31);
                        T right = __shfl_sync(0xffffffffu, c.x, (lane + 1) & 31);
                        if constexpr (N > 128) {
                            if (lane == 0) left = el[a];
                            if (lane == 31) right = er[a];
                        }
                        dx[a][0] = c.y - left;
                        dx[a][1] = c.z - c.x;
                        dx[a][2] = c.w - c.y;
                        dx[a][3] = right - c.z;
                        dy[a][0] = ap[a].x - am[a].x;
                        dy[a][1] = ap[a].y - am[a].y;
                        dy[a][2] = ap[a].z - am[a].z;
                        dy[a][3] = ap[a].w - am[a].w;
                        dz[a][0] = au[a].x - ad[a].x;
                        dz[a][1] = au[a].y - ad[a].y;
                        dz[a][2] = au[a].z - ad[a].z;
                        dz[a][3] = au[a].w - ad[a].w;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        T q = dx[0][r] + dy[0][r];
                        if (!INCR) q -= (dx[1][r] + dy[1][r]) * inv_rho;
                        q += dz[0][r];
                        if (!INCR) q -= dz[1][r] * inv_rho;
                        o[r] = -q * half_n;
                    }
                }
                stage[(x >> 1) * S + l] = V{o[0], o[1]};  // z_m = r_{2m} + i r_{2m+1}
                stage[((x >> 1) + 1) * S + l] = V{o[2], o[3]};
            }
        } else {
            for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
                const int l = idx >> X::LOGN;
                const int x = idx & (N - 1);
                const int y = y0 + l;
                const Idx v = (Idx)line0 * N + idx;
                const Idx xp = v + (x + 1 == N ? 1 - N : 1), xm = v + (x == 0 ? N - 1 : -1);
                const Idx yp = v + (y + 1 == N ? (1 - N) * sn : sn), ym = v + (y == 0 ? (N - 1) * sn : -sn);
                T q = (F_c0[xp] - F_c0[xm]) + (F_c1[yp] - F_c1[ym]);
                if (!INCR) q -= ((L_c0[xp] - L_c0[xm]) + (L_c1[yp] - L_c1[ym])) * inv_rho;
                q += F_c2[v + zp] - F_c2[v + zm];
                if (!INCR) q -= (L_c2[v + zp] - L_c2[v + zm]) * inv_rho;
                stage_r[((x >> 1) * S + l) * 2 + (x & 1)] = -q * half_n;  // z_m = r_{2m} + i r_{2m+1}
            }
        }
        __syncthreads();
        V xr[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) xr[r] = stage[(jt + TT * r) * S + lt];
        col_fft<H, false, 2, S>(xr, buf, s_tw, jt, lt);
        __syncthreads();  // col_fft's last readers are done with both buffers
#pragma unroll
        for (int r = 0; r < 8; ++r) stage[(jt + TT * r) * S + lt] = xr[r];
        __syncthreads();
        V* S_c = Sp + (long long)c * (Vn / 2);
        for (int idx = threadIdx.x; idx < LPB * H; idx += blockDim.x) {
            const int l = idx >> (X::LOGN - 1);
            const int kk = idx & (H - 1);
            const int line = line0 + l;
            if (line >= nlines) continue;
            const V Zk = stage[kk * S + l];
            V out;
            if (kk == 0) {
                out = V{Zk.x + Zk.y, Zk.x - Zk.y};  // (X_0, X_{N/2}) packed
            } else {
                const V Zc = cconj(stage[(H - kk) * S + l]);
                const V E = cscale(cadd(Zk, Zc), T(0.5));
                const V O = cscale(mul_mi(csub(Zk, Zc)), T(0.5));
                out = cadd(E, cmul(s_tw[kk], O));
            }
            S_c[(long long)line * H + kk] = out;
        }
    }
}

template <typename T, typename TO, int N, int D, bool INCR>
__device__ __forceinline__ void xinv_fixed_tile(const Launch& L, int bid, bool& twl) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    using X = XPlan<N>;
    constexpr int H = X::H, LPB = X::LPB, S = X::S, TT = ColPlan<H>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    T* S0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* S1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    TO* O0 = INCR ? (TO*)L.U64[0] : (TO*)Args::U(L, 0);
    TO* O1 = INCR ? (TO*)L.U64[1] : (TO*)Args::U(L, 1);
    T* __restrict__ DUout = (T*)L.D32;
    if (ctrl->done) return;
    constexpr long long Vn = (D == 3) ? (long long)N * N * N : (long long)N * N;
    constexpr int nlines = (D == 3) ? N * N : N;
    const int par = (int)(ctrl->k & 1);
    V* Sp = reinterpret_cast<V*>(INCR ? S0 : (par ? S0 : S1));
    TO* Out = par ? O0 : O1;
    const TO* In = par ? O1 : O0;
    // u~ as float pairs (Ctrl::u_pair), as in xinv_tile
    const bool upair = INCR && ctrl->u_pair;
    const float* Plo_in = INCR ? reinterpret_cast<const float*>(par ? L.U64[0] : L.U64[1]) + D * Vn : nullptr;
    float* Plo_out = INCR ? reinterpret_cast<float*>(par ? L.U64[1] : L.U64[0]) + D * Vn : nullptr;
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* buf = s_tw + N;
    V* stage = buf + H * S;
    if (!twl) {  // exp(-2 pi i m / N) depends on N only: loaded on the block's first tile
        load_twiddles(s_tw, Args::tw(L), N);
        twl = true;
    }
    constexpr int NB = nlines / LPB;  // one component per tile, as in xfwd_fixed_tile
    const int c0 = bid / NB;
    const int line0 = (bid % NB) * LPB;
    const int lt = threadIdx.x % LPB, jt = threadIdx.x / LPB;
    for (int c = c0; c < c0 + 1; ++c) {
        V* S_c = Sp + (long long)c * (Vn / 2);
        // the low parts of u~_k this thread updates at the end, loaded now so that their
        // latency overlaps the transform (LPB * N = 4096: four groups of four x per thread)
        float4 lo_k[4];
        if constexpr (INCR && std::is_same<T, float>::value) {
            if (upair) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = (threadIdx.x + q * kFftThreads) * 4;
                    const int line = line0 + (e >> X::LOGN);
                    lo_k[q] = line < nlines ? *reinterpret_cast<const float4*>(
                                                  Plo_in + (long long)c * Vn + (long long)line * N + (e & (N - 1)))
                                            : float4{0.f, 0.f, 0.f, 0.f};
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < LPB * H; idx += blockDim.x) {
            const int l = idx >> (X::LOGN - 1);
            const int kk = idx & (H - 1);
            const int line = line0 + l;
            V Z = V{T(0), T(0)};
            if (line < nlines) {
                const V Xk = S_c[(long long)line * H + kk];
                if (kk == 0) {
                    Z = V{T(0.5) * (Xk.x + Xk.y), T(0.5) * (Xk.x - Xk.y)};
                } else {
                    const V Xc = cconj(S_c[(long long)line * H + (H - kk)]);
                    const V E = cscale(cadd(Xk, Xc), T(0.5));
                    const V O = cmul(cscale(csub(Xk, Xc), T(0.5)), cconj(s_tw[kk]));
                    Z = cadd(E, mul_i(O));
                }
            }
            stage[kk * S + l] = Z;
        }
        __syncthreads();
        V xr[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) xr[r] = stage[(jt + TT * r) * S + lt];
        col_fft<H, true, 2, S>(xr, buf, s_tw, jt, lt);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; ++r) stage[(jt + TT * r) * S + lt] = xr[r];
        __syncthreads();
        const T* stage_r = reinterpret_cast<const T*>(stage);
        TO* O_c = Out + (long long)c * Vn;
        const TO* I_c = In + (long long)c * Vn;
        if constexpr (std::is_same<T, float>::value) {
            // four consecutive x per thread (two staged complex values): one float4 store,
            // or for the increment two double2 read-modify-writes and a float4 store of the
            // increment (fields are 256-byte aligned, x and N multiples of 4)
            static_assert(LPB * N / 4 == 4 * kFftThreads, "four groups of four x per thread");
            auto store = [&](int q) {
                const int idx = threadIdx.x + q * kFftThreads;
                const int e = idx * 4;
                const int l = e >> X::LOGN;
                const int xi = e & (N - 1);
                const int line = line0 + l;
                if (line < nlines) {
                    const V a = stage[(xi >> 1) * S + l];
                    const V b = stage[((xi >> 1) + 1) * S + l];
                    const long long o = (long long)line * N + xi;
                    if constexpr (INCR) {
                        static_assert(std::is_same<TO, double>::value, "increment accumulates in double");
                        if (upair) {
                            const float4 p = lo_k[q];
                            *reinterpret_cast<float4*>(Plo_out + (long long)c * Vn + o) =
                                float4{p.x + a.x, p.y + a.y, p.z + b.x, p.w + b.y};
                        } else {
                            const double2 i0 = *reinterpret_cast<const double2*>(I_c + o);
                            const double2 i1 = *reinterpret_cast<const double2*>(I_c + o + 2);
                            *reinterpret_cast<double2*>(O_c + o) = double2{i0.x + (TO)a.x, i0.y + (TO)a.y};
                            *reinterpret_cast<double2*>(O_c + o + 2) = double2{i1.x + (TO)b.x, i1.y + (TO)b.y};
                        }
                        *reinterpret_cast<float4*>(DUout + (long long)c * Vn + o) = float4{a.x, a.y, b.x, b.y};
                    } else if constexpr (std::is_same<TO, float>::value) {
                        *reinterpret_cast<float4*>(O_c + o) = float4{a.x, a.y, b.x, b.y};
                    } else {
                        *reinterpret_cast<double2*>(O_c + o) = double2{(TO)a.x, (TO)a.y};
                        *reinterpret_cast<double2*>(O_c + o + 2) = double2{(TO)b.x, (TO)b.y};
                    }
                }
            };
            // unrolled where the prefetched low parts of u~ live in registers; the plain
            // float pass runs faster rolled
            if constexpr (INCR) {
#pragma unroll
                for (int q = 0; q < 4; ++q) store(q);
            } else {
#pragma unroll 1
                for (int q = 0; q < 4; ++q) store(q);
            }
        } else {
            for (int idx = threadIdx.x; idx < LPB * N; idx += blockDim.x) {
                const int l = idx >> X::LOGN;
                const int xi = idx & (N - 1);
                const int line = line0 + l;
                if (line < nlines) {
                    const T v = stage_r[((xi >> 1) * S + l) * 2 + (xi & 1)];
                    const long long o = (long long)line * N + xi;
                    if (INCR) {
                        if (upair)
                            Plo_out[(long long)c * Vn + o] = Plo_in[(long long)c * Vn + o] + (float)v;
                        else
                            O_c[o] = I_c[o] + (TO)v;
                        DUout[(long long)c * Vn + o] = v;
                    } else {
                        O_c[o] = (TO)v;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ fused inverse y + x passes (3D float, N = 128)
// The inverse y and x transforms of one z-plane of one component in one block: the plane's
// 64 columns take faxis_fixed_tile's inverse y transform (AXIS 1, MODE 1) in four rounds
// of 16, into a shared plane (128 y rows of 64 x-frequencies, pitch 66) instead of back to
// the spectrum in L2; then xinv_fixed_tile's four groups of 32 lines take their
// complex-to-real transforms from it.  Same arithmetic in the same order as the two
// separate passes (the same bits), with one L2 round trip of the spectrum and one launch
// less per iteration.  While a group's x transform runs, that group's plane rows (32 x 66
// values) hold its buffer (64 frequencies x 33 lines, XPlan's padded stride).  68.6 KB of
// shared memory: 3 blocks per SM, one wave for the 384 planes of a 128^3 cell.  Tiles are
// those of the x passes (tiles_x, 1536 per RVE); tiles 384 and up have nothing to do.
// (The forward counterpart, the x transforms of a plane's lines followed by the y
// transforms of its columns, ran slower than the two separate passes and is not used.)
struct PlaneFused {
    static constexpr int N = 128, H = 64, P = 66, LPB = 32, S = 33, G = N / LPB;
};

template <typename TO, bool INCR>
__device__ __forceinline__ void yxinv_tile(const Launch& L, int bid, bool& twl) {
    using T = float;
    using V = float2;
    using Args = FftArgs<T>;
    using X = XPlan<128>;
    using PF = PlaneFused;
    constexpr int N = PF::N, H = PF::H, P = PF::P, LPB = PF::LPB, S = PF::S, TT = ColPlan<H>::T;
    if (bid >= 3 * N) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    if (ctrl->done) return;
    T* S0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* S1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    TO* O0 = INCR ? (TO*)L.U64[0] : (TO*)Args::U(L, 0);
    TO* O1 = INCR ? (TO*)L.U64[1] : (TO*)Args::U(L, 1);
    T* __restrict__ DUout = (T*)L.D32;
    constexpr long long Vn = (long long)N * N * N;
    const int par = (int)(ctrl->k & 1);
    V* Sp = reinterpret_cast<V*>(INCR ? S0 : (par ? S0 : S1));
    TO* Out = par ? O0 : O1;
    const TO* In = par ? O1 : O0;
    const bool upair = INCR && ctrl->u_pair;  // u~ as float pairs (Ctrl::u_pair)
    const float* Plo_in = INCR ? reinterpret_cast<const float*>(par ? L.U64[0] : L.U64[1]) + 3 * Vn : nullptr;
    float* Plo_out = INCR ? reinterpret_cast<float*>(par ? L.U64[1] : L.U64[0]) + 3 * Vn : nullptr;
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* plane = s_tw + N;
    if (!twl) {  // exp(-2 pi i m / N) depends on N only: loaded on the block's first tile
        load_twiddles(s_tw, Args::tw(L), N);
        twl = true;
    }
    const int c = bid / N, z = bid % N;
    // inverse y transforms of the plane's columns, 16 at a time (faxis_fixed_tile, AXIS 1,
    // MODE 1), into the shared plane
    using CP = ColPlan<N>;
    {
        const int cl = threadIdx.x % CP::TK, j = threadIdx.x / CP::TK;
        const V* S_c = Sp + (long long)c * (Vn / 2) + (long long)z * N * H;
        for (int k0 = 0; k0 < H; k0 += CP::TK) {
            V x[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) x[r] = S_c[(long long)(j + CP::T * r) * H + k0 + cl];
            col_fft<N, true, 1, P, true>(x, plane + k0, s_tw, j, cl);
            __syncthreads();  // the transform's last readers of these columns are done
#pragma unroll
            for (int r = 0; r < 8; ++r) plane[(j + CP::T * r) * P + k0 + cl] = x[r];
        }
    }
    const int lt = threadIdx.x % LPB, jt = threadIdx.x / LPB;
    TO* O_c = Out + (long long)c * Vn;
    const TO* I_c = In + (long long)c * Vn;
    for (int g = 0; g < PF::G; ++g) {
        V* gr = plane + g * LPB * P;
        const int line0 = z * N + g * LPB;
        float4 lo_k[4];  // low parts of u~_k for the final update (see xinv_fixed_tile)
        if constexpr (INCR) {
            if (upair) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = (threadIdx.x + q * kFftThreads) * 4;
                    lo_k[q] = *reinterpret_cast<const float4*>(Plo_in + (long long)c * Vn +
                                                               (long long)(line0 + (e >> X::LOGN)) * N + (e & (N - 1)));
                }
            }
        }
        __syncthreads();  // the plane is complete / the previous group's readers are done
        // complex-to-real split of the group's rows into registers, then into its x buffer
        V zz[LPB * H / kFftThreads];
#pragma unroll
        for (int i = 0; i < LPB * H / kFftThreads; ++i) {
            const int idx = threadIdx.x + i * kFftThreads;
            const int l = idx >> (X::LOGN - 1);
            const int kk = idx & (H - 1);
            const V Xk = gr[l * P + kk];
            if (kk == 0) {
                zz[i] = V{T(0.5) * (Xk.x + Xk.y), T(0.5) * (Xk.x - Xk.y)};
            } else {
                const V Xc = cconj(gr[l * P + (H - kk)]);
                const V E = cscale(cadd(Xk, Xc), T(0.5));
                const V O = cmul(cscale(csub(Xk, Xc), T(0.5)), cconj(s_tw[kk]));
                zz[i] = cadd(E, mul_i(O));
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < LPB * H / kFftThreads; ++i) {
            const int idx = threadIdx.x + i * kFftThreads;
            gr[(idx & (H - 1)) * S + (idx >> (X::LOGN - 1))] = zz[i];
        }
        __syncthreads();
        V xr[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) xr[r] = gr[(jt + TT * r) * S + lt];
        col_fft<H, true, 2, S, true>(xr, gr, s_tw, jt, lt);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; ++r) gr[(jt + TT * r) * S + lt] = xr[r];
        __syncthreads();
        // four consecutive x per thread (xinv_fixed_tile's float stores)
        auto store = [&](int q) {
            const int idx = threadIdx.x + q * kFftThreads;
            const int e = idx * 4;
            const int l = e >> X::LOGN;
            const int xi = e & (N - 1);
            const int line = line0 + l;
            const V a = gr[(xi >> 1) * S + l];
            const V b = gr[((xi >> 1) + 1) * S + l];
            const long long o = (long long)line * N + xi;
            if constexpr (INCR) {
                if (upair) {
                    const float4 p = lo_k[q];
                    *reinterpret_cast<float4*>(Plo_out + (long long)c * Vn + o) =
                        float4{p.x + a.x, p.y + a.y, p.z + b.x, p.w + b.y};
                } else {
                    const double2 i0 = *reinterpret_cast<const double2*>(I_c + o);
                    const double2 i1 = *reinterpret_cast<const double2*>(I_c + o + 2);
                    *reinterpret_cast<double2*>(O_c + o) = double2{i0.x + (TO)a.x, i0.y + (TO)a.y};
                    *reinterpret_cast<double2*>(O_c + o + 2) = double2{i1.x + (TO)b.x, i1.y + (TO)b.y};
                }
                *reinterpret_cast<float4*>(DUout + (long long)c * Vn + o) = float4{a.x, a.y, b.x, b.y};
            } else {
                *reinterpret_cast<float4*>(O_c + o) = float4{a.x, a.y, b.x, b.y};
            }
        };
        if constexpr (INCR) {
#pragma unroll
            for (int q = 0; q < 4; ++q) store(q);
        } else {
#pragma unroll 1
            for (int q = 0; q < 4; ++q) store(q);
        }
    }
}

// faxis_tile with a fixed column length N (see ColPlan); same tiles and modes.
template <typename T, int N, int D, int AXIS, int MODE, bool INCR>
__device__ __forceinline__ void faxis_fixed_tile(const Launch& L, int bid, bool& twl) {
    using V = typename Cx<T>::t;
    using Args = FftArgs<T>;
    using P = ColPlan<N>;
    constexpr int H = N / 2, TK = P::TK, TT = P::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Ctrl* __restrict__ ctrl = L.ctrl;
    T* U0 = INCR ? (T*)L.S32 : Args::U(L, 0);
    T* U1 = INCR ? (T*)L.S32 : Args::U(L, 1);
    const V* __restrict__ g_tw = Args::tw(L);
    const T* __restrict__ ksq = Args::ksq(L);
    const T scale = Args::scale(L);
    if (ctrl->done) return;
    constexpr long long Vn = (D == 3) ? (long long)N * N * N : (long long)N * N;
    const int par = (int)(ctrl->k & 1);
    V* S = reinterpret_cast<V*>(par ? U0 : U1);
    V* s_tw = reinterpret_cast<V*>(smem_raw);
    V* buf = s_tw + N;
    if (!twl) {  // exp(-2 pi i m / N) depends on N only: loaded on the block's first tile
        load_twiddles(s_tw, g_tw, N);
        twl = true;
    }
    constexpr int gxa = H / TK;
    constexpr int gya = (D == 3) ? N : 1;
    const int col0 = (bid % gxa) * TK;
    const int outer = (bid / gxa) % gya;
    const int c = bid / (gxa * gya);
    long long base;
    constexpr long long es_g = (D == 3 && AXIS == 2) ? (long long)N * H : H;
    if (D == 3 && AXIS == 1)
        base = (long long)c * (Vn / 2) + (long long)outer * N * H + col0;
    else if (D == 3 && AXIS == 2)
        base = (long long)c * (Vn / 2) + (long long)outer * H + col0;
    else
        base = (long long)c * (Vn / 2) + col0;
    const int cl = threadIdx.x % TK;
    const int j = threadIdx.x / TK;
    // the change of the solved spectrum for r_d (float phase, see Launch::Sprev): the kept
    // u^_k is kept in tile order (the same tile and thread hold a mode every iteration:
    // rows of 256 values, not the spectrum's column stride) and copied asynchronously
    // into the block's second shared buffer while the forward transform runs
    constexpr bool kSpec = MODE == 2 && !INCR && D == 3 && AXIS == 2 && std::is_same<T, float>::value;
    float2* __restrict__ Sp = kSpec ? reinterpret_cast<float2*>(L.Sprev) : nullptr;
    const bool have = kSpec && Sp && ctrl->spec_have;
    float2* pre = reinterpret_cast<float2*>(buf + N * TK);
    if constexpr (kSpec) {
        if (have) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
                cp_async8(pre + r * kFftThreads + threadIdx.x, Sp + ((long long)bid * 8 + r) * kFftThreads + threadIdx.x);
            cp_async_commit();
        }
    }
    float acc = 0.f;
    V x[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = S[base + (j + TT * r) * es_g + cl];
    if (MODE == 1) {
        col_fft<N, true, 1, TK, true>(x, buf, s_tw, j, cl);
    } else {
        col_fft<N, false, 1, TK, true>(x, buf, s_tw, j, cl);
        if (MODE == 2) {
            const T kout = (D == 3) ? __ldg(ksq + outer) : T(0);
            const T kcol = __ldg(ksq + min(col0 + cl, H - 1)) + kout;
            if constexpr (kSpec) {
                if (have) cp_async_wait_all();  // this thread's own copies
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const T den = __ldg(ksq + j + TT * r) + kcol;
                x[r] = cscale(x[r], den > T(0) ? scale / den : T(0));
                if constexpr (kSpec) {
                    if (Sp) {
                        const long long at = ((long long)bid * 8 + r) * kFftThreads + threadIdx.x;
                        if (have) {
                            const float2 o = pre[r * kFftThreads + threadIdx.x];
                            const float dx = x[r].x - o.x, dy = x[r].y - o.y;
                            acc += den * (dx * dx + dy * dy);
                        }
                        Sp[at] = x[r];
                    }
                }
            }
            col_fft<N, true, 1, TK, true>(x, buf, s_tw, j, cl);
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) S[base + (j + TT * r) * es_g + cl] = x[r];
    if constexpr (kSpec) {
        if (Sp) {
            // the spectrum holds x-frequencies 0 .. N/2-1, the first packed with N/2: the
            // others stand for their conjugate partners too (weight 2); the tile's sum goes
            // to its own slot (summed in a fixed order by the local pass)
            __shared__ float s_red[kFftThreads / 32];
            acc *= (col0 + cl == 0) ? 1.f : 2.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < kFftThreads / 32; ++w) t += (double)s_red[w];
                L.zpart[bid] = t;
                if (bid == 0) {
                    Ctrl* c = const_cast<Ctrl*>(ctrl);
                    c->spec_sum = ctrl->spec_have;
                    c->spec_next = 1;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ launch

inline int lines_per_block(int n, int nlines) {
    int lpb = 2048 / n;
    if (lpb < 1) lpb = 1;
    if (lpb > nlines) lpb = nlines;
    return lpb;
}

template <typename T, int D, bool INCR>
__global__ void __launch_bounds__(kFftThreads)
k_xfwd(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    const void* twp = nullptr;  // the twiddle table in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        xfwd_tile<T, D, INCR>(rds[tl.x], tl.y, twp);
        __syncthreads();
    }
}

template <typename T, typename TO, int D, bool INCR>
__global__ void __launch_bounds__(kFftThreads)
k_xinv(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    const void* twp = nullptr;  // the twiddle table in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        xinv_tile<T, TO, D, INCR>(rds[tl.x], tl.y, twp);
        __syncthreads();
    }
}

template <typename T, int D, int AXIS, int MODE, bool INCR>
__global__ void __launch_bounds__(kFftThreads)
k_faxis(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    const void* twp = nullptr;  // the twiddle table in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        faxis_tile<T, D, AXIS, MODE, INCR>(rds[tl.x], tl.y, twp);
        __syncthreads();
    }
}

// 3 blocks of 68.6 KB per SM (one wave of a 128^3 cell's 384 planes): at most 85 registers
template <typename TO, bool INCR>
__global__ void __launch_bounds__(kFftThreads, 3) k_yxinv128(const Launch* __restrict__ rds,
                                                          const int2* __restrict__ tiles, int ntiles) {
    bool twl = false;  // the twiddle table is in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        yxinv_tile<TO, INCR>(rds[tl.x], tl.y, twl);
        __syncthreads();
    }
}

constexpr size_t kPlaneSmem = (size_t)(PlaneFused::N + PlaneFused::N * PlaneFused::P) * sizeof(float2);

// The float z solve, which also keeps the spectrum for r_d, is held to 64 registers (4
// blocks per SM): with 73 registers and 3 blocks it runs 2 us slower per 128^3 pass.
template <typename T, int N, int D, int AXIS, int MODE, bool INCR>
__global__ void __launch_bounds__(kFftThreads, (MODE == 2 && !INCR && std::is_same<T, float>::value) ? 4 : 1)
k_faxis_fixed(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    bool twl = false;  // the twiddle table is in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        faxis_fixed_tile<T, N, D, AXIS, MODE, INCR>(rds[tl.x], tl.y, twl);
        __syncthreads();
    }
}

template <typename T, int N, int D, bool INCR>
__global__ void __launch_bounds__(kFftThreads)
k_xfwd_fixed(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    bool twl = false;  // the twiddle table is in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        xfwd_fixed_tile<T, N, D, INCR>(rds[tl.x], tl.y, twl);
        __syncthreads();
    }
}

template <typename T, typename TO, int N, int D, bool INCR>
__global__ void __launch_bounds__(kFftThreads)
k_xinv_fixed(const Launch* __restrict__ rds, const int2* __restrict__ tiles, int ntiles) {
    bool twl = false;  // the twiddle table is in shared memory
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tl = tiles[t];
        xinv_fixed_tile<T, TO, N, D, INCR>(rds[tl.x], tl.y, twl);
        __syncthreads();
    }
}

template <typename T, int N>
constexpr size_t xfixed_smem() {
    return (size_t)(N + 2 * XPlan<N>::H * XPlan<N>::S) * sizeof(typename Cx<T>::t);
}

template <typename T, int N, int D = 3, int AXIS = 1, int MODE = 0, bool INCR = false>
constexpr size_t fixed_smem() {
    // one transform buffer; the float z solve adds the buffer of the kept spectrum's copies
    constexpr bool spec = MODE == 2 && !INCR && D == 3 && AXIS == 2 && std::is_same<T, float>::value;
    return (size_t)(N + (spec ? 2 : 1) * N * ColPlan<N>::TK) * sizeof(typename Cx<T>::t);
}

template <typename K>
void go(K kern, const Exec& E, int cls, size_t smem) {
    const int nt = E.ntiles[cls];
    const int grid = persistent_grid((const void*)kern, kFftThreads, smem, nt);
    kern<<<grid, kFftThreads, smem, E.stream>>>(E.rds, E.tiles[cls], nt);
}

// y/z pass: the fixed-length kernel when every member of the launch is a 3D grid of
// N in {128, 256, 512} with the fixed kernel's column tile, else the general one.
template <typename T, int D, int AXIS, int MODE, bool INCR>
void go_axis(const Exec& E, int cls, size_t sma) {
    const int tk = std::is_same<T, double>::value ? E.rep->tk64 : E.rep->tk32;
    if constexpr (D == 3) {
        switch (E.uniform_geom ? E.uniform_n : 0) {
            case 128:
                if (tk == ColPlan<128>::TK)
                    return go(k_faxis_fixed<T, 128, D, AXIS, MODE, INCR>, E, cls,
                              fixed_smem<T, 128, D, AXIS, MODE, INCR>());
                break;
            case 256:
                if (tk == ColPlan<256>::TK)
                    return go(k_faxis_fixed<T, 256, D, AXIS, MODE, INCR>, E, cls,
                              fixed_smem<T, 256, D, AXIS, MODE, INCR>());
                break;
            case 512:
                if (tk == ColPlan<512>::TK)
                    return go(k_faxis_fixed<T, 512, D, AXIS, MODE, INCR>, E, cls,
                              fixed_smem<T, 512, D, AXIS, MODE, INCR>());
                break;
            default:
                break;
        }
    }
    go(k_faxis<T, D, AXIS, MODE, INCR>, E, cls, sma);
}

// x passes: the fixed-length kernels under the same conditions (3D, one N of 128, 256
// or 512 for every member, lines per block of the fixed kernels).
template <typename T, int D, bool INCR>
void go_xfwd(const Exec& E, size_t smx) {
    if constexpr (D == 3) {
        const int lpb = E.rep->lpb;
        switch (E.uniform_geom ? E.uniform_n : 0) {
            case 128:
                if (lpb == XPlan<128>::LPB) return go(k_xfwd_fixed<T, 128, D, INCR>, E, kTilesX, xfixed_smem<T, 128>());
                break;
            case 256:
                if (lpb == XPlan<256>::LPB) return go(k_xfwd_fixed<T, 256, D, INCR>, E, kTilesX, xfixed_smem<T, 256>());
                break;
            case 512:
                if (lpb == XPlan<512>::LPB) return go(k_xfwd_fixed<T, 512, D, INCR>, E, kTilesX, xfixed_smem<T, 512>());
                break;
            default:
                break;
        }
    }
    go(k_xfwd<T, D, INCR>, E, kTilesX, smx);
}

template <typename T, typename TO, int D, bool INCR>
void go_xinv(const Exec& E, size_t smx) {
    if constexpr (D == 3) {
        const int lpb = E.rep->lpb;
        switch (E.uniform_geom ? E.uniform_n : 0) {
            case 128:
                if (lpb == XPlan<128>::LPB)
                    return go(k_xinv_fixed<T, TO, 128, D, INCR>, E, kTilesX, xfixed_smem<T, 128>());
                break;
            case 256:
                if (lpb == XPlan<256>::LPB)
                    return go(k_xinv_fixed<T, TO, 256, D, INCR>, E, kTilesX, xfixed_smem<T, 256>());
                break;
            case 512:
                if (lpb == XPlan<512>::LPB)
                    return go(k_xinv_fixed<T, TO, 512, D, INCR>, E, kTilesX, xfixed_smem<T, 512>());
                break;
            default:
                break;
        }
    }
    go(k_xinv<T, TO, D, INCR>, E, kTilesX, smx);
}

// stage < 0: all passes of one iteration; otherwise only pass `stage`
// (3D: 0 x-forward, 1 y-forward, 2 z solve, 3 y-inverse, 4 x-inverse;
//  2D: 0 x-forward, 1 y solve, 2 x-inverse).  INCR: the float increment
// projection of the double polish (see launch_fft_incr).
// the float passes of 3D grids of N = 128 with the fixed kernels' geometry fuse the inverse
// y and x transforms of each z-plane (yxinv_tile)
bool fused_xy(const Exec& E) {
    return E.rep->dim == 3 && E.uniform_geom && E.uniform_n == 128 && E.rep->lpb == XPlan<128>::LPB &&
           E.rep->tk32 == ColPlan<128>::TK;
}

template <typename T, int D, bool INCR>
cudaError_t run_fft(const Exec& E, int stage) {
    const int f = std::is_same<T, double>::value ? 1 : 0;
    const int ax = f ? kTilesAx64 : kTilesAx32;
    const size_t smx = E.smem_x[f], sma = E.smem_a[f];
    const int last = D == 3 ? 4 : 2;
    auto want = [&](int s) { return stage < 0 || stage == s; };
    static_assert(!INCR || std::is_same<T, float>::value, "increment projection runs in float");
    bool finv = false;  // inverse y and x passes of a z-plane fused in one block
    if constexpr (D == 3 && std::is_same<T, float>::value) finv = fused_xy(E);
    if (want(0)) go_xfwd<T, D, INCR>(E, smx);
    if constexpr (D == 3) {
        if (want(1)) go_axis<T, D, 1, 0, INCR>(E, ax, sma);
        if (want(2)) go_axis<T, D, 2, 2, INCR>(E, ax, sma);
        if (!finv && want(3)) go_axis<T, D, 1, 1, INCR>(E, ax, sma);
    } else if (want(1)) {
        go_axis<T, D, 1, 2, INCR>(E, ax, sma);
    }
    if (finv && want(last)) {
        if constexpr (D == 3 && std::is_same<T, float>::value) {
            if constexpr (INCR)
                go(k_yxinv128<double, true>, E, kTilesX, kPlaneSmem);
            else
                go(k_yxinv128<float, false>, E, kTilesX, kPlaneSmem);
        }
    } else if (want(last)) {
        if constexpr (INCR)
            go_xinv<float, double, D, true>(E, smx);
        else
            go_xinv<T, T, D, false>(E, smx);
    }
    return cudaGetLastError();
}

template <typename T, int D>
cudaError_t set_smem_attrs(int bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (r != cudaSuccess) e = r;
    };
    set((const void*)k_xfwd<T, D, false>);
    set((const void*)k_xinv<T, T, D, false>);
    if constexpr (std::is_same<T, float>::value && D == 3) {
        set((const void*)k_yxinv128<float, false>);
        set((const void*)k_yxinv128<double, true>);
    }
    set((const void*)k_faxis<T, D, 1, 0, false>);
    set((const void*)k_faxis<T, D, 1, 1, false>);
    set((const void*)k_faxis<T, D, 1, 2, false>);
    set((const void*)k_faxis<T, D, 2, 2, false>);
    if constexpr (D == 3) {
        auto fixed = [&](auto tag) {
            constexpr int N = decltype(tag)::value;
            set((const void*)k_xfwd_fixed<T, N, D, false>);
            set((const void*)k_xinv_fixed<T, T, N, D, false>);
            if constexpr (std::is_same<T, float>::value) {
                set((const void*)k_xfwd_fixed<float, N, D, true>);
                set((const void*)k_xinv_fixed<float, double, N, D, true>);
            }
            set((const void*)k_faxis_fixed<T, N, D, 1, 0, false>);
            set((const void*)k_faxis_fixed<T, N, D, 1, 1, false>);
            set((const void*)k_faxis_fixed<T, N, D, 2, 2, false>);
            if constexpr (std::is_same<T, float>::value) {
                set((const void*)k_faxis_fixed<T, N, D, 1, 0, true>);
                set((const void*)k_faxis_fixed<T, N, D, 1, 1, true>);
                set((const void*)k_faxis_fixed<T, N, D, 2, 2, true>);
            }
        };
        fixed(std::integral_constant<int, 128>());
        fixed(std::integral_constant<int, 256>());
        fixed(std::integral_constant<int, 512>());
    }
    if constexpr (std::is_same<T, float>::value) {
        set((const void*)k_xfwd<float, D, true>);
        set((const void*)k_xinv<float, double, D, true>);
        set((const void*)k_faxis<float, D, 1, 0, true>);
        set((const void*)k_faxis<float, D, 1, 1, true>);
        set((const void*)k_faxis<float, D, 1, 2, true>);
        set((const void*)k_faxis<float, D, 2, 2, true>);
    }
    return e;
}

}  // namespace

cudaError_t launch_fft(const Exec& E, bool fp64, int stage) {
    const int dim = E.rep->dim;
    if (fp64) return dim == 3 ? run_fft<double, 3, false>(E, stage) : run_fft<double, 2, false>(E, stage);
    return dim == 3 ? run_fft<float, 3, false>(E, stage) : run_fft<float, 2, false>(E, stage);
}

bool fft_stage_empty(const Exec& E, bool fp64, int stage) {
    return !fp64 && fused_xy(E) && stage == 3;
}

cudaError_t launch_fft_incr(const Exec& E, int stage) {
    return E.rep->dim == 3 ? run_fft<float, 3, true>(E, stage) : run_fft<float, 2, true>(E, stage);
}

// Radix sequence for a transform length L = 2^a 3^b: radix 8 first, then 4, 2, 3.
int factor_radices(int L, int* rad) {
    int np = 0;
    while (L % 8 == 0) { rad[np++] = 8; L /= 8; }
    if (L % 4 == 0) { rad[np++] = 4; L /= 4; }
    if (L % 2 == 0) { rad[np++] = 2; L /= 2; }
    while (L % 3 == 0) { rad[np++] = 3; L /= 3; }
    return L == 1 ? np : -1;
}

namespace {
std::mutex g_geo_mu;
std::map<std::pair<int, int>, Geometry> g_geo;  // (dim, n) -> tuned geometry
}  // namespace

void register_geometry(int dim, int n, const Geometry& g) {
    std::lock_guard<std::mutex> lock(g_geo_mu);
    g_geo[{dim, n}] = g;
}

bool lookup_geometry(int dim, int n, Geometry* g) {
    std::lock_guard<std::mutex> lock(g_geo_mu);
    auto it = g_geo.find({dim, n});
    if (it == g_geo.end()) return false;
    *g = it->second;
    return true;
}

Geometry default_geometry(int dim, int n) {
    Geometry g{};
    const int H = n / 2;
    const int nlines = dim == 3 ? n * n : n;
    // small grids: fewer lines / columns per block until a pass has ~2 blocks per SM
    const int want_blocks = 2 * 152;
    g.lpb = lines_per_block(n, nlines);
    while (g.lpb > 1 && (nlines + g.lpb - 1) / g.lpb < want_blocks) g.lpb /= 2;
    auto ax_blocks = [&](int tk) { return ((H + tk - 1) / tk) * (dim == 3 ? n : 1) * dim; };
    g.tk64 = FftArgs<double>::tk < H ? FftArgs<double>::tk : H;
    g.tk32 = FftArgs<float>::tk < H ? FftArgs<float>::tk : H;
    while (g.tk64 > 1 && ax_blocks(g.tk64) < want_blocks) g.tk64 /= 2;
    while (g.tk32 > 1 && ax_blocks(g.tk32) < want_blocks) g.tk32 /= 2;
    if (dim == 3 && (n == 128 || n == 256 || n == 512)) {  // the fixed-length kernels' tiles
        g.tk64 = g.tk32 = 2048 / n;
        g.lpb = 4096 / n;
    }
    g.np_half = factor_radices(H, g.rad_half);
    g.np_full = factor_radices(n, g.rad_full);
    return g;
}

void apply_geometry(Launch& L, const Geometry& g) {
    const int n = L.n;
    const int nlines = L.dim == 3 ? n * n : n;
    L.lpb = g.lpb < nlines ? g.lpb : nlines;
    L.xblocks = (nlines + L.lpb - 1) / L.lpb;
    L.tk64 = g.tk64;
    L.tk32 = g.tk32;
    L.plan.n = n;
    L.plan.np_half = g.np_half;
    L.plan.np_full = g.np_full;
    for (int i = 0; i < kMaxPasses; ++i) {
        L.plan.rad_half[i] = i < g.np_half ? g.rad_half[i] : 0;
        L.plan.rad_full[i] = i < g.np_full ? g.rad_full[i] : 0;
    }
    // per-pass divisors; the twiddle table has N entries, so a transform of
    // length Lt = N / twmul steps through it with stride twmul Lt / (Ns R) = N / (Ns R)
    auto passes = [n](int Lt, const int* rad, int np, FftPass* out) {
        int Ns = 1;
        for (int p = 0; p < kMaxPasses; ++p) {
            const int R = p < np ? rad[p] : 1;
            out[p].nb = make_fastdiv((unsigned)(Lt / R));
            out[p].ns = make_fastdiv((unsigned)Ns);
            out[p].tstep = n / (Ns * R);
            if (p < np) Ns *= R;
        }
    };
    passes(n / 2, L.plan.rad_half, g.np_half, L.plan.pass_half);
    passes(n, L.plan.rad_full, g.np_full, L.plan.pass_full);
    L.plan.div_n = make_fastdiv((unsigned)n);
    L.plan.div_h = make_fastdiv((unsigned)(n / 2));
    L.plan.div_tk64 = make_fastdiv((unsigned)L.tk64);
    L.plan.div_tk32 = make_fastdiv((unsigned)L.tk32);
}

void set_geometry(Launch& L) {
    L.half_n64 = 0.5 * (double)L.n;
    L.scale64 = 2.0 / (double)L.V;
    L.two_nsq64 = 2.0 * (double)L.n * (double)L.n;
    L.half_n32 = (float)L.half_n64;
    L.scale32 = (float)L.scale64;
    L.two_nsq32 = (float)L.two_nsq64;
    // voxels a local tile covers per sweep: a whole block of threads, or fewer for small
    // cells so that the local step still spreads over ~2 blocks per SM (a function of the
    // RVE's size only, so results do not depend on what else runs in the launch)
    int chunk = kLocalThreads;
    while (chunk > 32 && (L.V + chunk - 1) / chunk < 2 * 152) chunk /= 2;
    L.local_chunk = chunk;
    const long long want = (L.V + chunk - 1) / chunk;
    const long long cap = kLocalTileCap;
    L.local_blocks = (int)(want < cap ? want : cap);
    Geometry g;
    if (!lookup_geometry(L.dim, L.n, &g)) g = default_geometry(L.dim, L.n);
    apply_geometry(L, g);
}

int tiles_local(const Launch& L) { return L.local_blocks; }
// the fixed-length x kernels (3D, N = 128, 256, 512 with their lines per block) take one
// component per tile
int tiles_x(const Launch& L) {
    const bool fixed = L.dim == 3 && ((L.n == 128 && L.lpb == XPlan<128>::LPB) ||
                                      (L.n == 256 && L.lpb == XPlan<256>::LPB) ||
                                      (L.n == 512 && L.lpb == XPlan<512>::LPB));
    return L.xblocks * (fixed ? L.dim : 1);
}
int tiles_ax(const Launch& L, bool fp64) {
    const int H = L.n / 2;
    const int tk = fp64 ? L.tk64 : L.tk32;
    return ((H + tk - 1) / tk) * (L.dim == 3 ? L.n : 1) * L.dim;
}

size_t smem_x_bytes(const Launch& L, bool fp64) {
    const size_t v = fp64 ? sizeof(double2) : sizeof(float2);
    return (size_t)L.n * v + 2 * (size_t)L.lpb * (L.n / 2) * v;
}
size_t smem_a_bytes(const Launch& L, bool fp64) {
    const size_t v = fp64 ? sizeof(double2) : sizeof(float2);
    return (size_t)L.n * v + 2 * (size_t)L.n * (fp64 ? L.tk64 : L.tk32) * v;
}

int persistent_grid(const void* kernel, int threads, size_t smem, int ntiles) {
    static std::mutex mu;
    static std::map<std::pair<const void*, size_t>, int> cache;
    static int sms = 0;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (sms == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
        }
        auto it = cache.find({kernel, smem});
        if (it != cache.end()) {
            per_sm = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
                per_sm <= 0)
                per_sm = 1;
            cache[{kernel, smem}] = per_sm;
        }
    }
    const long long cap = (long long)per_sm * sms;
    if (ntiles < 1) return 1;
    return (int)(ntiles < cap ? ntiles : cap);
}

// Allow the FFT kernels the dynamic shared memory the largest grid needs.
cudaError_t prepare_fft_kernels(int n) {
    (void)n;
    const int bytes = 200 * 1024;
    cudaError_t e;
    if ((e = set_smem_attrs<double, 2>(bytes)) != cudaSuccess) return e;
    if ((e = set_smem_attrs<double, 3>(bytes)) != cudaSuccess) return e;
    if ((e = set_smem_attrs<float, 2>(bytes)) != cudaSuccess) return e;
    return set_smem_attrs<float, 3>(bytes);
}

}  // namespace admm
