// Device-side building blocks of the resistive-MHD IMEX stage (arXiv 2110.03732).
//
// Everything here is evaluated in the local orthonormal frame of the conformally
// flat metric gamma_ij = psi^4 delta_ij (beta^i = 0): a vector X^i has orthonormal
// components X_hat = psi^2 X^i, a covector X_hat = psi^-2 X_i, so that every dot and
// cross product is the flat-space one.  Densitised conserved variables are
// q_D = psi^6 D, q_S = psi^8 S_hat, q_tau = psi^6 tau, q_E = psi^4 E_hat,
// q_B = psi^4 B_hat (Sec. 2.1 with sqrt(gamma) = psi^6 and sqrt(gamma_hat) = 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dword.cuh"

namespace grmhd {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FIXED = 2 };

// Unsigned 32-bit division by a run-time invariant d >= 1 through a multiply-high
// (Granlund & Montgomery, PLDI 1994, the unsigned form exact for every 32-bit
// dividend): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// t / d = (h + ((t - h) >> min(l, 1))) >> max(l - 1, 0), h = umulhi(t, m).  The
// compiler's own division by a run-time value goes through float reciprocals and
// conversions, which on GB300 share the FP64 pipe with the implicit solve.
struct FastDiv {
    unsigned m, d;
    int s1, s2;
};

inline FastDiv make_fastdiv(unsigned d)
{
    int l = 0;
    while (l < 32 && (1ull << l) < d) l++;
    FastDiv f;
    f.d = d;
    f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l - 1 > 0 ? l - 1 : 0;
    return f;
}

__host__ __device__ __forceinline__ unsigned fdiv(unsigned t, const FastDiv& f)
{
#ifdef __CUDA_ARCH__
    const unsigned h = __umulhi(t, f.m);
#else
    const unsigned h = (unsigned)(((unsigned long long)t * f.m) >> 32);
#endif
    return (h + ((t - h) >> f.s1)) >> f.s2;
}

// Padded grid, passed by value to every kernel.  Active directions have ng = 2 ghost
// cells per side; inactive ones have one cell and no ghosts.  Arrays are x-fastest.
struct Dims {
    int n[3], ng[3], N[3], bc[3], act[3];
    long long st[3];       // strides of x, y, z
    double idx[3];         // 1/dx (0 where inactive)
    double gh;             // Gamma_hat_1 = Gamma/(Gamma - 1)
    double igh;            // 1/Gamma_hat_1
    long long ncell;       // padded cells
    FastDiv dv[2];         // division by n[0] and by n[1] (interior cell index -> i, j, k)
    FastDiv dvp[2];        // division by n[d] + 1 (1 where inactive): face and edge indices
    int mk[3];             // march length along d (faces or edges per thread)
    FastDiv dq[3];         // division by the chunks per line along d, (n[d] + mk[d]) / mk[d]
    float hix[3][2];       // 1/(2 dx) as a double-word hi + lo (the FP32 flux divergence)
};

// set the march length along d (and its chunk divisor) of a launch's copy of the grid
inline void set_march(Dims& g, int d, int K)
{
    g.mk[d] = K;
    g.dq[d] = make_fastdiv((unsigned)((g.n[d] + K) / K));
}

// the divisors of a grid whose extents n, act and idx are set (march length 1
// everywhere), and the double-word split of 1/(2 dx)
inline void set_divisors(Dims& g)
{
    for (int d = 0; d < 2; d++) {
        g.dv[d] = make_fastdiv((unsigned)g.n[d]);
        g.dvp[d] = make_fastdiv((unsigned)(g.act[d] ? g.n[d] + 1 : 1));
    }
    for (int d = 0; d < 3; d++) {
        set_march(g, d, 1);
        const double h = 0.5 * g.idx[d];
        g.hix[d][0] = (float)h;
        g.hix[d][1] = (float)(h - (double)g.hix[d][0]);
    }
}

// (i0, i1, i2) of index t over an x-fastest box whose first two extents have the
// divisors f0, f1 (t < 2^32)
__device__ __forceinline__ void box_coords(long long t, const FastDiv& f0, const FastDiv& f1, int* idx)
{
    const unsigned tt = (unsigned)t;
    const unsigned q0 = fdiv(tt, f0);
    const unsigned q1 = fdiv(q0, f1);
    idx[0] = (int)(tt - q0 * f0.d);
    idx[1] = (int)(q0 - q1 * f1.d);
    idx[2] = (int)q1;
}

// padded coordinates of interior cell t (x fastest); t < 2^32 (the library refuses
// grids of 2^32 or more interior cells)
__device__ __forceinline__ void interior_coords(const Dims& g, long long t, int* c)
{
    box_coords(t, g.dv[0], g.dv[1], c);
#pragma unroll
    for (int d = 0; d < 3; d++) c[d] += g.ng[d];
}

struct P8 { double* p[8]; };          // rho, u^1..3, p, E^1..3  (or 8 conserved)
struct P3 { double* p[3]; };          // three face / edge / R arrays
struct CP8 { const double* p[8]; };
struct CP3 { const double* p[3]; };

// ---------------------------------------------------------------------------
// boundary conditions applied on read: periodic wraps, outflow clamps to the last
// interior cell (last real face for a face along its own direction), fixed reads
// the stored ghost value
// ---------------------------------------------------------------------------

// (m - lo) mod n for m - lo in [-2n, 3n): stencil indices stay within a few cells of the
// interior and a periodic direction has n >= 2, so two conditional shifts each way
// suffice (an integer % by a run-time n goes through float reciprocals and conversions
// that share the FP64 pipe)
__device__ __forceinline__ int wrap_periodic(int m, int lo, int n)
{
    int r = m - lo;
    r += r < 0 ? n : 0;
    r += r < 0 ? n : 0;
    r -= r >= n ? n : 0;
    r -= r >= n ? n : 0;
    return lo + r;
}

__device__ __forceinline__ int map_cell(const Dims& g, int d, int m)
{
    if (!g.act[d]) return 0;
    const int lo = g.ng[d], n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) return wrap_periodic(m, lo, n);
    if (g.bc[d] == BC_OUTFLOW) return m < lo ? lo : (m > lo + n - 1 ? lo + n - 1 : m);
    return m;
}

__device__ __forceinline__ int map_face(const Dims& g, int d, int m)
{
    if (!g.act[d]) return 0;
    const int lo = g.ng[d], n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) return wrap_periodic(m, lo, n);
    if (g.bc[d] == BC_OUTFLOW) return m < lo ? lo : (m > lo + n ? lo + n : m);
    return m;
}

// Bounds-checked builds (-DGRMHD_CHECK_BOUNDS, the library's checked copy): every
// array index made by lin() or by an explicit stride offset passes through chk(),
// which counts an index outside [0, ncell) in a per-translation-unit device counter
// and redirects it to index 0, so that the access stays inside the array and the
// kernel runs on; grmhd_bounds_violations reads and clears the counters.  In the
// normal build chk() is the identity.
#ifdef GRMHD_CHECK_BOUNDS
static __device__ unsigned long long g_oob_count;
#endif

__device__ __forceinline__ long long chk(const Dims& g, long long i)
{
#ifdef GRMHD_CHECK_BOUNDS
    if (i < 0 || i >= g.ncell) {
        atomicAdd(&g_oob_count, 1ull);
        return 0;
    }
#else
    (void)g;
#endif
    return i;
}

// host side: this translation unit's counter (0 in the normal build); reset clears it
#ifdef GRMHD_CHECK_BOUNDS
#define GRMHD_OOB_READER(name)                                                                  \
    unsigned long long name(bool reset)                                                         \
    {                                                                                           \
        unsigned long long v = 0;                                                               \
        if (cudaMemcpyFromSymbol(&v, g_oob_count, sizeof v) != cudaSuccess) return ~0ull;       \
        if (reset) {                                                                            \
            const unsigned long long z = 0;                                                     \
            if (cudaMemcpyToSymbol(g_oob_count, &z, sizeof z) != cudaSuccess) return ~0ull;     \
        }                                                                                       \
        return v;                                                                               \
    }
#else
#define GRMHD_OOB_READER(name) \
    unsigned long long name(bool) { return 0; }
#endif

__device__ __forceinline__ long long lin(const Dims& g, int i, int j, int k)
{
    return chk(g, (long long)i + g.st[1] * j + g.st[2] * k);
}

// mapped cell index of padded coordinates c[3]
__device__ __forceinline__ long long cell_at(const Dims& g, const int* c)
{
    return lin(g, map_cell(g, 0, c[0]), map_cell(g, 1, c[1]), map_cell(g, 2, c[2]));
}

// mapped index of the face array of direction fd at padded coordinates c[3]
__device__ __forceinline__ long long face_at(const Dims& g, int fd, const int* c)
{
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; d++) m[d] = (d == fd) ? map_face(g, d, c[d]) : map_cell(g, d, c[d]);
    return lin(g, m[0], m[1], m[2]);
}

// discrete divergence of the staggered q_B at the interior cell with padded
// coordinates c and linear index o (Sec. 3.2): sum over the active directions of
// (upper face - lower face) / dx; the upper face is mapped by the boundary rule
__device__ __forceinline__ double cell_divb(const Dims& g, const double* const* bf, const int* c, long long o)
{
    double dv = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!g.act[d]) continue;
        int cu[3] = {c[0], c[1], c[2]};
        cu[d] += 1;
        dv += (bf[d][face_at(g, d, cu)] - bf[d][o]) * g.idx[d];
    }
    return dv;
}

template <typename T, int K>
__device__ __forceinline__ T scale_pow2(T v);

// cell-centred q_B^e of the cell at padded coordinates c: the cell is mapped first,
// then the mean of its two e-faces (the lower face alone where the upper one lies
// outside a fixed-boundary array; the halving on the integer pipe); an inactive e
// stores the cell value itself
__device__ __forceinline__ double cell_qB(const Dims& g, const double* __restrict__ bf, int e, const int* c)
{
    int m[3];
#pragma unroll
    for (int d = 0; d < 3; d++) m[d] = map_cell(g, d, c[d]);
    const long long i0 = lin(g, m[0], m[1], m[2]);
    if (!g.act[e]) return bf[i0];
    int h = m[e] + 1;
    if (g.bc[e] == BC_PERIODIC && h == g.ng[e] + g.n[e]) h = g.ng[e];
    if (h >= g.N[e]) return bf[i0];
    const long long i1 = chk(g, i0 + (long long)(h - m[e]) * g.st[e]);
    return scale_pow2<double, -1>(bf[i0] + bf[i1]);
}

// ---------------------------------------------------------------------------
// MC limiter (monotonised central, van Leer 1974)
//
// The half slope used for a face state is 1/2 minmod(2 d-, (d- + d+)/2, 2 d+)
// = minmod(d-, (u+ - u-)/4, d+) exactly (the factors are powers of two).  minmod is
// evaluated on the IEEE bit patterns with integer instructions: the three arguments
// agree in sign when their sign bits agree, and among same-signed doubles the one
// of least magnitude has the least 63-bit magnitude field.  GB300's FP64 pipe is the
// bottleneck of this path, so keeping compares and selects off it matters.
// ---------------------------------------------------------------------------

template <typename T> struct Bits;
template <> struct Bits<double> {
    using I = long long;
    static __device__ __forceinline__ I to(double x) { return __double_as_longlong(x); }
    static __device__ __forceinline__ double from(I i) { return __longlong_as_double(i); }
    static constexpr I MAG = 0x7fffffffffffffffLL;
};
template <> struct Bits<float> {
    using I = int;
    static __device__ __forceinline__ I to(float x) { return __float_as_int(x); }
    static __device__ __forceinline__ float from(I i) { return __int_as_float(i); }
    static constexpr I MAG = 0x7fffffff;
};

// v * 2^K.  In FP64, exactly, by moving the exponent field on the integer pipe (a
// multiply by a power of two would take an FP64 issue slot): normal values stay exact,
// a result below the normal range (|v| < 2^-1020 for K = -2) flushes to a signed zero,
// one above it becomes a signed infinity, and infinities and NaN pass unchanged.  In
// FP32 the multiply itself (the FP32 pipe has room to spare).
template <typename T, int K>
__device__ __forceinline__ T scale_pow2(T v)
{
    if (sizeof(T) == 4) return v * (K >= 0 ? T(1 << (K >= 0 ? K : 0)) : T(1) / T(1 << (K < 0 ? -K : 0)));
    using I = typename Bits<T>::I;
    constexpr int MB = sizeof(T) == 8 ? 52 : 23;
    constexpr I EMAX = sizeof(T) == 8 ? 2047 : 255;
    const I b = Bits<T>::to(v);
    const I e = (b >> MB) & EMAX;
    const I sgn = b & ~Bits<T>::MAG;
    const I moved = b + (I(K) << MB);
    const I r = (e == EMAX) ? b : ((e != 0 && e + K >= 1) ? (e + K < EMAX ? moved : (sgn | (EMAX << MB))) : sgn);
    return Bits<T>::from(r);
}

template <typename T>
__device__ __forceinline__ T minmod3(T a, T b, T c)
{
    using I = typename Bits<T>::I;
    const I ia = Bits<T>::to(a), ib = Bits<T>::to(b), ic = Bits<T>::to(c);
    const I ma = ia & Bits<T>::MAG, mb = ib & Bits<T>::MAG, mc = ic & Bits<T>::MAG;
    I r = ma <= mb ? ia : ib;
    const I mr = ma <= mb ? ma : mb;
    r = mr <= mc ? r : ic;
    // sign bits differ somewhere -> 0 (signed zeros of agreeing sign give that zero)
    return ((ia ^ ib) | (ia ^ ic)) < 0 ? T(0) : Bits<T>::from(r);
}

// left/right states at the face between a1 and a2 from the four cells a0 a1 a2 a3
template <typename T>
__device__ __forceinline__ void mc_face(T a0, T a1, T a2, T a3, T& L, T& R)
{
    const T dm = a1 - a0, d0 = a2 - a1, dp = a3 - a2;
    L = a1 + minmod3<T>(dm, scale_pow2<T, -2>(a2 - a0), d0);
    R = a2 - minmod3<T>(d0, scale_pow2<T, -2>(a3 - a1), dp);
}

// 1/sqrt(x) through CUDA's reciprocal square root, in the precision of x (for the
// stencil kernels' 1 + u^2 the FP64 form counts as many FP64 instructions as
// rsqrt_ge1 below)
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// PPM (Colella & Woodward 1984: interface interpolation with the MC slope and the
// monotonicity limits of the parabola, no steepening or flattening).  a[0..5] are the
// cells c-3..c+2; L is the right edge of cell c-1, R the left edge of cell c.
// the MC slope of cell a0 (twice the half slope minmod(D-, (a+ - a-)/4, D+))
template <typename T>
__device__ __forceinline__ T ppm_slope(T am, T a0, T ap)
{
    return scale_pow2<T, 1>(minmod3<T>(a0 - am, scale_pow2<T, -2>(ap - am), ap - a0));
}

// the interface value between cells a0 and ap with slopes s0, s1
template <typename T>
__device__ __forceinline__ T ppm_iface_s(T a0, T ap, T s0, T s1)
{
    return a0 + T(0.5) * (ap - a0) - (s1 - s0) * T(1.0 / 6.0);
}

template <typename T>
__device__ __forceinline__ T ppm_iface(T am, T a0, T ap, T app)
{
    return ppm_iface_s<T>(a0, ap, ppm_slope<T>(am, a0, ap), ppm_slope<T>(a0, ap, app));
}

// signs of a product from the IEEE bit patterns (an FP64 multiply and compare would
// take two FP64 issue slots): x y > 0 when both are nonzero with equal signs, x y < 0
// when both are nonzero with opposite signs
template <typename T>
__device__ __forceinline__ bool prod_pos(T x, T y)
{
    using I = typename Bits<T>::I;
    const I bx = Bits<T>::to(x), by = Bits<T>::to(y);
    return (bx ^ by) >= 0 && (bx & Bits<T>::MAG) != 0 && (by & Bits<T>::MAG) != 0;
}

template <typename T>
__device__ __forceinline__ bool prod_neg(T x, T y)
{
    using I = typename Bits<T>::I;
    const I bx = Bits<T>::to(x), by = Bits<T>::to(y);
    return (bx ^ by) < 0 && (bx & Bits<T>::MAG) != 0 && (by & Bits<T>::MAG) != 0;
}

// Colella & Woodward's monotonicity limits of the parabola through aL, a0, aR: flat
// at a local extremum ((aR - a0)(a0 - aL) <= 0), else the edge whose overshoot the
// parabola would take past the other is moved (dd m6 > dd^2, or -dd^2 > dd m6, with
// dd = aR - aL and m6 = 6 (a0 - (aL + aR)/2)).  The comparisons are decided as signs:
// dd m6 - dd^2 = 2 dd t1 and dd m6 + dd^2 = 2 dd t2 with t1 = 3 a0 - aL - 2 aR and
// t2 = 3 a0 - 2 aL - aR, and the moved edges are 3 a0 - 2 aR = t1 + aL and
// 3 a0 - 2 aL = t2 + aR.  Where rounding could flip a decision the two outcomes
// coincide (t1 = 0 moves aL onto itself), so the limiter stays continuous.
template <typename T>
__device__ __forceinline__ void ppm_limit(T a0, T& aL, T& aR)
{
    if (!prod_pos(aR - a0, a0 - aL)) {
        aL = a0;
        aR = a0;
        return;
    }
    const T dd = aR - aL;
    const T t1 = T(3) * a0 - aL - T(2) * aR, t2 = T(3) * a0 - T(2) * aL - aR;
    if (prod_pos(dd, t1)) aL = t1 + aL;
    else if (prod_neg(dd, t2)) aR = t2 + aR;
}

template <typename T>
__device__ __forceinline__ void ppm_face(const T* a, T& L, T& R)
{
    const T im = ppm_iface<T>(a[0], a[1], a[2], a[3]);
    const T i0 = ppm_iface<T>(a[1], a[2], a[3], a[4]);
    const T ip = ppm_iface<T>(a[2], a[3], a[4], a[5]);
    T lL = im, lR = i0, rL = i0, rR = ip;
    ppm_limit<T>(a[2], lL, lR);
    ppm_limit<T>(a[3], rL, rR);
    L = lR;
    R = rL;
}

// coordinate m along d brought inside the padded array: the PPM stencil reaches one
// cell past the two stored ghost layers, where periodic wraps, outflow takes the
// boundary cell and fixed the outermost stored ghost.  Inside the array m is kept.
__device__ __forceinline__ int ext_cell(const Dims& g, int d, int m)
{
    if (!g.act[d] || (m >= 0 && m < g.N[d])) return m;
    const int lo = g.ng[d], n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) return wrap_periodic(m, lo, n);
    if (g.bc[d] == BC_OUTFLOW) return m < lo ? lo : lo + n - 1;
    return m < 0 ? 0 : g.N[d] - 1;
}

// fused multiply-add in the precision of its operands
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------------------
// physical state at a face in the orthonormal frame (Sec. 2.1)
// ---------------------------------------------------------------------------

template <typename T>
struct FaceStateT {
    T q[8];    // densitised conserved: D, S_1..3, tau, E^1..3
    T f[8];    // flux of the same along the face normal
    T iW;      // 1/W of the state
};
using FaceState = FaceStateT<double>;

// prim: rho, u^1..3, p, E^1..3 (coordinate components) and B^1..3 (coordinate);
// psi, alpha at the face; d = normal direction.  T = double on the FP64 path, float
// for the reconstruction and fluxes of the mixed-precision path.
template <typename T>
__device__ __forceinline__ void face_state(const T* pr, const T* B, int d, T psi, T alp, T gh, FaceStateT<T>& s)
{
    const T p2 = psi * psi, p4 = p2 * p2, p6 = p4 * p2;
    const T rho = pr[0], p = pr[4];
    T u[3], E[3], Bh[3];
#pragma unroll
    for (int i = 0; i < 3; i++) { u[i] = p2 * pr[1 + i]; E[i] = p2 * pr[5 + i]; Bh[i] = p2 * B[i]; }
    // W and 1/W from one reciprocal square root (no division)
    const T x = T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T iW = rsqrt_t(x);
    const T W = x * iW;
    s.iW = iW;
    const T rhoh = rho + gh * p;
    const T D = rho * W;
    const T U = T(0.5) * (E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + Bh[0] * Bh[0] + Bh[1] * Bh[1] + Bh[2] * Bh[2]);
    T S[3];
    S[0] = rhoh * W * u[0] + (E[1] * Bh[2] - E[2] * Bh[1]);
    S[1] = rhoh * W * u[1] + (E[2] * Bh[0] - E[0] * Bh[2]);
    S[2] = rhoh * W * u[2] + (E[0] * Bh[1] - E[1] * Bh[0]);
    const T tau = rhoh * W * W - p + U - D;
    s.q[0] = p6 * D;
#pragma unroll
    for (int j = 0; j < 3; j++) s.q[1 + j] = p6 * p2 * S[j];
    s.q[4] = p6 * tau;
#pragma unroll
    for (int j = 0; j < 3; j++) s.q[5 + j] = p4 * E[j];
    // fluxes along d (beta = 0), with W v = u: D v^d = rho u^d and
    // rho h W^2 v^d v^j = rho h u^d u^j
    const T Dv = rho * u[d];
    const T rhu = rhoh * u[d];
    s.f[0] = p4 * alp * Dv;
#pragma unroll
    for (int j = 0; j < 3; j++)
        s.f[1 + j] = p6 * alp * ((j == d ? p + U : T(0)) + rhu * u[j] - E[d] * E[j] - Bh[d] * Bh[j]);
    s.f[4] = p4 * alp * (S[d] - Dv);
    // (f_E^j)^d = alpha psi^2 eta^{djk} B_hat_k
    const T ap2 = alp * p2;
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    s.f[5 + d] = T(0);
    s.f[5 + d1] = ap2 * Bh[d2];
    s.f[5 + d2] = -ap2 * Bh[d1];
}

// One side's half of the unit-speed HLL flux in flat space (psi = alpha = 1), in the
// orthonormal frame: g = f + SG q, SG = +1 for the left state and -1 for the right, so
// that f_L + f_R - (q_R - q_L) = g_L + g_R with q and f as in face_state.  Grouping by
// state lets shared factors merge: with a = u^d + SG W,
//   D:     rho u^d + SG rho W                                  = rho a
//   S_j:   (p + U) delta_dj + rho h u^d u^j - E^d E^j - B^d B^j
//          + SG (rho h W u^j + (E x B)_j)                      = rho h a u^j + ...
//   tau:   S_d - rho u^d + SG (rho h W^2 - p + U - rho W)
//   E^j:   eta^{djk} B_k + SG E^j
// pr: rho, u^1..3, p, E^1..3; B: the three components; iW gets 1/W of the state.
template <typename T, int SG>
__device__ __forceinline__ void face_hll_half(const T* pr, const T* B, int d, T gh, T* g, T& iW)
{
    const T s = T(SG);
    const T rho = pr[0], p = pr[4];
    const T u[3] = {pr[1], pr[2], pr[3]};
    const T E[3] = {pr[5], pr[6], pr[7]};
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    const T x = T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    iW = rsqrt_t(x);
    const T W = x * iW;
    const T rhoh = rho + gh * p;
    const T hW = rhoh * W;
    // 2U = |E|^2 + |B|^2; p + U and U - p each as one fused multiply-add
    const T U2 = E[0] * E[0] + E[1] * E[1] + E[2] * E[2] + B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const T Xd = E[d1] * B[d2] - E[d2] * B[d1];   // (E x B)_d, used twice
    const T a = u[d] + s * W;
    const T K = rhoh * a;
    g[0] = rho * a;
    // S_j halves, j != d: the component (E x B)_j = E^{j+1} B^{j+2} - E^{j+2} B^{j+1} is
    // used once, so it enters the chain of fused multiply-adds directly
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if (j == d) continue;
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        g[1 + j] = fma_t(K, u[j], fma_t(-E[d], E[j], fma_t(-B[d], B[j], fma_t(s * E[j1], B[j2], -(s * E[j2]) * B[j1]))));
    }
    // S_d: K u^d + (p + U - E^d E^d - B^d B^d) + SG (E x B)_d
    g[1 + d] = fma_t(K, u[d], fma_t(-E[d], E[d], fma_t(-B[d], B[d], fma_t(T(0.5), U2, p))) + s * Xd);
    // tau: S_d - rho u^d + SG (rho h W^2 - p + U - rho W)
    //    = S_d + SG (h W W + U - p) - rho a,  and rho a is g[0]
    const T Sd = fma_t(hW, u[d], Xd);
    const T Tq = fma_t(W, hW, fma_t(T(0.5), U2, -p));
    g[4] = (Sd + s * Tq) - g[0];
    g[5 + d] = s * E[d];
    g[5 + d1] = B[d2] + s * E[d1];
    g[5 + d2] = s * E[d2] - B[d1];
}

// binary64 <-> binary32 on the integer pipe.  On GB300 the hardware conversions (F2F)
// issue on the FP64 pipe at the rate of an FP64 add, and the implicit solve is bound
// by that pipe; these re-bias the exponent field (1023 <-> 127) and move the mantissa
// with integer instructions, and take no hardware conversion on any path (a rare
// fallback would still be predicated into every call).  d2f rounds the 29 dropped
// mantissa bits half away from zero (IEEE round-to-nearest-even differs only at exact
// ties); below the normal binary32 range it flushes to a signed zero, above it gives
// a signed infinity, and NaN stays NaN.  f2d is exact for normal floats and zero,
// flushes binary32 denormals to a signed zero and keeps infinities and NaN.  Used for
// the FP32 and double-word copies of the Newton solve, where only the size of the
// rounding matters.
__device__ __forceinline__ float d2f_int(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned sgn = hi & 0x80000000u;
    const unsigned f = (sgn | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
    const unsigned big = nan ? (sgn | 0x7fc00000u) : (sgn | 0x7f800000u);
    return __uint_as_float(e - 897u <= 253u ? f : (e < 897u ? sgn : big));
}

__device__ __forceinline__ double f2d_int(float v)
{
    const unsigned f = __float_as_uint(v);
    const unsigned e = (f >> 23) & 0xffu;
    const unsigned sgn = f & 0x80000000u;
    const unsigned nhi = sgn | ((e + 896u) << 20) | ((f >> 3) & 0xfffffu);
    const unsigned shi = e == 0u ? sgn : (sgn | 0x7ff00000u | ((f & 0x7fffffu) ? 0x80000u : 0u));
    const bool normal = e - 1u < 254u;
    return __hiloint2double((int)(normal ? nhi : shi), (int)(normal ? (f << 29) : 0u));
}

// a value of the stencil precision T widened to FP64 for storing: FP32 on the integer
// pipe (exact for normal floats and zero; a denormal float is stored as zero)
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_int(x); }

// an FP64 metric factor (psi, alpha) in the stencil precision T: itself, or rounded to
// binary32 on the integer pipe (a metric stencil converts tens of them per face or
// edge, and a hardware conversion would issue each on the FP64 pipe); mean2 = (a + b)/2
// in T (FP64: the sum first; FP32: of the two rounded values, no FP64 instruction).
// Face fields and constants, a few per face, keep the hardware conversion: the FP32
// kernels leave the FP64 pipe idle, and it is fewer instructions.
template <typename T> __device__ __forceinline__ T met_t(double x);
template <> __device__ __forceinline__ double met_t<double>(double x) { return x; }
template <> __device__ __forceinline__ float met_t<float>(double x) { return d2f_int(x); }
template <typename T> __device__ __forceinline__ T mean2(double a, double b);
template <> __device__ __forceinline__ double mean2<double>(double a, double b) { return 0.5 * (a + b); }
template <> __device__ __forceinline__ float mean2<float>(double a, double b)
{
    return 0.5f * (d2f_int(a) + d2f_int(b));
}

constexpr unsigned kHi1e30 = 0x46293E59u;   // high word of 1e30 (a start beyond is discarded)

// FP64 tests on the integer pipe (an FP64 compare also issues on the FP64 pipe):
// x is finite; x > 0 (false for NaN and +inf); |x| < a bound given by its high word
// (within 2^-20, from below)
__device__ __forceinline__ bool finite_int(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool pos_int(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool mag_below_int(double x, unsigned bound_hi)
{
    return ((unsigned)__double2hiint(x) & 0x7fffffffu) < bound_hi;
}

// 1/sqrt(x) for 1 <= x < 2^127 and 1/x for x > 0 in FP64 from an FP32 estimate y,
// each with one correction step of order three (the truncated binomial series).
// rsqrt: e = 1 - x y^2, 1/sqrt(x) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + ...);
// reciprocal: e = 1 - x y, 1/x = y / (1 - e) = y (1 + e + e^2 + ...).  The estimate
// is good to about 2^-21 (rsqrtf / __fdividef and the rounding of x to FP32), so the
// dropped terms are near 2^-63 and the result is within an ulp or so of the exact
// value: 5 FP64 instructions for rsqrt, 3 for the reciprocal, and none of the
// special-value branches of the library routines (their callers pass moderate
// positive values only).
__device__ __forceinline__ double rsqrt_ge1(double x)
{
    const double y = f2d_int(rsqrtf(d2f_int(x)));
    const double e = fma(-x, y * y, 1.0);
    return fma(y, e * fma(0.375, e, 0.5), y);
}

__device__ __forceinline__ double rcp_pos(double x)
{
    const double y = f2d_int(__fdividef(1.0f, d2f_int(x)));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/x for a positive x of moderate size in the stencil precision T (metric factors,
// speed products): rcp_pos in FP64, the division in FP32
__device__ __forceinline__ double rcp_t(double x) { return rcp_pos(x); }
__device__ __forceinline__ float rcp_t(float x) { return 1.0f / x; }

// ---------------------------------------------------------------------------
// implicit electric field + velocity solve (Sec. 2.4), xi = 0, orthonormal frame
// ---------------------------------------------------------------------------

struct CellIn {
    double D, S[3], tau, Es[3], B[3];   // undensitised orthonormal components
    double etat;                        // eta / (alpha a_ii dt); < 0: E held fixed
    double xi;                          // mean-field dynamo parameter (Sec. 2.2)
    double gh, igh;
    float ighf, xif;                    // FP32 copies of igh and xi (kernel constants)
    // set by cell_derive, once per cell: which E(u) applies, and the pieces of the
    // residual that do not depend on u
    int emode;                          // 0: E held fixed, 1: resistive, 2: with the dynamo
    double tD, B2h, Digh, etEs[3];      // tau + D, |B|^2 / 2, D / Gamma_hat, eta_t E*
};

__device__ __forceinline__ void cell_derive(CellIn& c)
{
    // E held fixed when eta_t < 0 or NaN; the dynamo form when xi != 0 (integer tests:
    // an FP64 compare issues on the FP64 pipe)
    const long long eb = __double_as_longlong(c.etat);
    const bool et_ok = (eb >= 0 && eb <= 0x7ff0000000000000ll) || eb == (long long)0x8000000000000000ull;
    c.emode = !et_ok ? 0 : ((__double_as_longlong(c.xi) << 1) != 0 ? 2 : 1);
    c.tD = c.tau + c.D;
    c.B2h = 0.5 * (c.B[0] * c.B[0] + c.B[1] * c.B[1] + c.B[2] * c.B[2]);
    c.Digh = c.D * c.igh;
#pragma unroll
    for (int i = 0; i < 3; i++) c.etEs[i] = c.etat * c.Es[i];
}

// A_k(W) of Sec. 2.4 for the dynamo parameter xi, and their W-derivatives:
//   A_0 = W + eta_t + xi^2 (W^2 - 1)/p,  A_1 = eta_t/q + xi^2 eta_t W/(p q),
//   A_2 = -xi eta_t/p,  A_3 = xi q/p,  A_4 = xi (1 - eta_t^2 + xi^2)/(p q),
//   A_5 = -1 - xi^2 W/p,  with p = W + eta_t, q = 1 + eta_t W
template <typename T>
struct DynT {
    T A[6], Ad[6];
};
using Dyn = DynT<double>;

template <typename T>
__device__ __forceinline__ void dyn_coeffs(T W, T et, T xi, DynT<T>& d, bool derivs)
{
    const T x2 = xi * xi, p = W + et, q = T(1) + et * W;
    const T ip = T(1) / p, iq = T(1) / q, ipq = ip * iq;
    d.A[0] = W + et + x2 * (W * W - T(1)) * ip;
    d.A[1] = et * iq + x2 * et * W * ipq;
    d.A[2] = -xi * et * ip;
    d.A[3] = xi * q * ip;
    d.A[4] = xi * (T(1) - et * et + x2) * ipq;
    d.A[5] = -T(1) - x2 * W * ip;
    if (derivs) {
        const T ip2 = ip * ip, iq2 = iq * iq;
        d.Ad[0] = T(1) + x2 * (T(1) + W * W + T(2) * W * et) * ip2;
        d.Ad[1] = -et * et * iq2 - x2 * et * et * (W * W - T(1)) * iq2 * ip2;
        d.Ad[2] = xi * et * ip2;
        d.Ad[3] = xi * (et * et - T(1)) * ip2;
        d.Ad[4] = -xi * (T(1) - et * et + x2) * (T(1) + et * et + T(2) * W * et) * iq2 * ip2;
        d.Ad[5] = -x2 * et * ip2;
    }
}

// dE_i/du_j with the dynamo (Sec. 2.4, orthonormal frame):
//   W A_0 dE_i/du_j = -A0' E_i u_j + A_1 W u_i E*_j + A3' B_i u_j + A_4 W u_i B_j
//     + (A_1 W delta_ij + A1' u_i u_j)(E*.u) + A_2 W eps_ijm E*_m + A2' (u x E*)_i u_j
//     + (A_4 W delta_ij + A4' u_i u_j)(B.u) + A_5 W eps_ijm B_m + A5' (u x B)_i u_j
template <typename T>
__device__ __forceinline__ void dE_dynamo(const T* A, const T* Ad, T W, const T* u, const T* E, const T* Es,
                                          const T* B, T dE[3][3])
{
    const T Esu = Es[0] * u[0] + Es[1] * u[1] + Es[2] * u[2];
    const T Bu = B[0] * u[0] + B[1] * u[1] + B[2] * u[2];
    const T uxEs[3] = {u[1] * Es[2] - u[2] * Es[1], u[2] * Es[0] - u[0] * Es[2], u[0] * Es[1] - u[1] * Es[0]};
    const T uxB[3] = {u[1] * B[2] - u[2] * B[1], u[2] * B[0] - u[0] * B[2], u[0] * B[1] - u[1] * B[0]};
    const T s = T(1) / (A[0] * W);
    const T dg = A[1] * W * Esu + A[4] * W * Bu;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            dE[i][j] = (-Ad[0] * E[i] * u[j] + A[1] * W * u[i] * Es[j] + Ad[3] * B[i] * u[j] + A[4] * W * u[i] * B[j] +
                        (Ad[1] * Esu + Ad[4] * Bu) * u[i] * u[j] + (Ad[2] * uxEs[i] + Ad[5] * uxB[i]) * u[j] +
                        (i == j ? dg : T(0))) * s;
    // A_2 W eps_ijm E*_m + A_5 W eps_ijm B_m
    const T X[3] = {(A[2] * Es[0] + A[5] * B[0]) * W * s, (A[2] * Es[1] + A[5] * B[1]) * W * s,
                    (A[2] * Es[2] + A[5] * B[2]) * W * s};
    dE[0][1] += X[2]; dE[0][2] -= X[1];
    dE[1][2] += X[0]; dE[1][0] -= X[2];
    dE[2][0] += X[1]; dE[2][1] -= X[0];
}

// |x| as the high word of its IEEE pattern with the sign cleared.  It is monotone in
// |x|, so integer maxima of these words give the largest magnitude to within 2^-20
// (relative, from below) without using the FP64 pipe.
__device__ __forceinline__ unsigned mag_hi(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
__device__ __forceinline__ double from_hi(unsigned h) { return __hiloint2double((int)h, 0); }

struct Eval {
    double W, iW, E[3], wt, U, A1, iWe, iden, Esu, f[3];
    double fm;   // max |f_i| (high-word maximum: within 2^-20 below the exact one)
    double M;    // momentum scale of f: max(|S_i|, |(E x B)_i|, |w_t u_i|), likewise
};

// E(u) from A_0 E = eta_t E* + A_1 (E*.u) u - u x B with A_0 = W + eta_t,
// A_1 = eta_t/(1 + eta_t W); then w_tilde and f = w_tilde u - S + E x B
__device__ __forceinline__ void evaluate(const CellIn& c, const double* u, Eval& e)
{
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double Wsq = 1.0 + uu;   // W^2
    e.iW = rsqrt_ge1(Wsq);
    e.W = Wsq * e.iW;
    if (c.emode == 2) {
        // A_0 E = eta_t E* + A_1 (E*.u) u + A_2 u x E* + A_3 B + A_4 (B.u) u + A_5 u x B
        Dyn dy;
        dyn_coeffs(e.W, c.etat, c.xi, dy, false);
        e.iWe = 1.0 / dy.A[0];
        e.A1 = dy.A[1];
        e.Esu = c.Es[0] * u[0] + c.Es[1] * u[1] + c.Es[2] * u[2];
        const double Bu = c.B[0] * u[0] + c.B[1] * u[1] + c.B[2] * u[2];
        const double a = dy.A[1] * e.Esu, b = dy.A[4] * Bu;
        const double uxEs[3] = {u[1] * c.Es[2] - u[2] * c.Es[1], u[2] * c.Es[0] - u[0] * c.Es[2],
                                u[0] * c.Es[1] - u[1] * c.Es[0]};
        const double uxB[3] = {u[1] * c.B[2] - u[2] * c.B[1], u[2] * c.B[0] - u[0] * c.B[2],
                               u[0] * c.B[1] - u[1] * c.B[0]};
#pragma unroll
        for (int i = 0; i < 3; i++)
            e.E[i] = (c.etat * c.Es[i] + (a + b) * u[i] + dy.A[2] * uxEs[i] + dy.A[3] * c.B[i] + dy.A[5] * uxB[i]) *
                     e.iWe;
    } else if (c.emode == 1) {
        // the three reciprocals 1/(W + eta_t), 1/(1 + eta_t W) and 1/(W^2 - 1/Gamma_hat)
        // from one division: r = 1/(a b d), 1/a = r b d, ...  (a, b >= 1 and d > 0, so
        // the product neither overflows nor cancels)
        const double a = e.W + c.etat, b = 1.0 + c.etat * e.W, d = Wsq - c.igh;
        const double ab = a * b, r = rcp_pos(ab * d);
        e.iWe = r * (b * d);
        e.A1 = c.etat * (r * (a * d));
        e.iden = r * ab;
        e.Esu = c.Es[0] * u[0] + c.Es[1] * u[1] + c.Es[2] * u[2];
        const double ae = e.A1 * e.Esu;
        e.E[0] = (c.etEs[0] + ae * u[0] - (u[1] * c.B[2] - u[2] * c.B[1])) * e.iWe;
        e.E[1] = (c.etEs[1] + ae * u[1] - (u[2] * c.B[0] - u[0] * c.B[2])) * e.iWe;
        e.E[2] = (c.etEs[2] + ae * u[2] - (u[0] * c.B[1] - u[1] * c.B[0])) * e.iWe;
    } else {
        e.iWe = 0.0; e.A1 = 0.0; e.Esu = 0.0;
        e.E[0] = c.Es[0]; e.E[1] = c.Es[1]; e.E[2] = c.Es[2];
    }
    e.U = 0.5 * (e.E[0] * e.E[0] + e.E[1] * e.E[1] + e.E[2] * e.E[2]) + c.B2h;
    if (c.emode != 1) e.iden = rcp_pos(Wsq - c.igh);
    e.wt = (e.W * (c.tD - e.U) - c.Digh) * e.iden;
    const double x0 = e.E[1] * c.B[2] - e.E[2] * c.B[1];
    const double x1 = e.E[2] * c.B[0] - e.E[0] * c.B[2];
    const double x2 = e.E[0] * c.B[1] - e.E[1] * c.B[0];
    const double w0 = e.wt * u[0], w1 = e.wt * u[1], w2 = e.wt * u[2];
    e.f[0] = w0 - c.S[0] + x0;
    e.f[1] = w1 - c.S[1] + x1;
    e.f[2] = w2 - c.S[2] + x2;
    e.fm = from_hi(max(mag_hi(e.f[0]), max(mag_hi(e.f[1]), mag_hi(e.f[2]))));
    e.M = from_hi(max(max(max(mag_hi(c.S[0]), mag_hi(c.S[1])), max(mag_hi(c.S[2]), mag_hi(x0))),
                      max(max(mag_hi(x1), mag_hi(x2)), max(mag_hi(w0), max(mag_hi(w1), mag_hi(w2))))));
}

// |f|^2 of an evaluated residual
__device__ __forceinline__ double fnorm2(const Eval& e) { return e.f[0] * e.f[0] + e.f[1] * e.f[1] + e.f[2] * e.f[2]; }

// Jacobian J_ij = w_t delta_ij + u_i dw_t/du_j + (dE/du_j x B)_i
__device__ __forceinline__ void jacobian(const CellIn& c, const double* u, const Eval& e, double J[3][3])
{
    const double iW = e.iW;
    double dE[3][3];   // dE_i / du_j
    if (c.emode == 2) {
        Dyn dy;
        dyn_coeffs(e.W, c.etat, c.xi, dy, true);
        dE_dynamo<double>(dy.A, dy.Ad, e.W, u, e.E, c.Es, c.B, dE);
    } else if (c.emode == 1) {
        // W (W + eta_t) dE_i/du_j = -E_i u_j + A_1 W u_i E*_j + (A_1 W delta_ij - A_1^2 u_i u_j)(E*.u)
        //                          - W eps_ijl B_l
        const double A1 = e.A1, a2 = A1 * A1 * e.Esu * iW;
        const double s = e.iWe;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                dE[i][j] = (-e.E[i] * u[j] * iW + A1 * u[i] * c.Es[j] - a2 * u[i] * u[j] +
                            (i == j ? A1 * e.Esu : 0.0)) * s;
        // - eps_ijl B_l / (W + eta_t)
        dE[0][1] -= c.B[2] * s; dE[0][2] += c.B[1] * s;
        dE[1][2] -= c.B[0] * s; dE[1][0] += c.B[2] * s;
        dE[2][0] -= c.B[1] * s; dE[2][1] += c.B[0] * s;
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) dE[i][j] = 0.0;
    }
    const double base = c.tD - e.U;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const double dU = e.E[0] * dE[0][j] + e.E[1] * dE[1][j] + e.E[2] * dE[2][j];
        const double dwt = (base * u[j] * iW - e.W * dU - 2.0 * e.wt * u[j]) * e.iden;
        // (dE/du_j x B)
        const double cx = dE[1][j] * c.B[2] - dE[2][j] * c.B[1];
        const double cy = dE[2][j] * c.B[0] - dE[0][j] * c.B[2];
        const double cz = dE[0][j] * c.B[1] - dE[1][j] * c.B[0];
        J[0][j] = u[0] * dwt + cx;
        J[1][j] = u[1] * dwt + cy;
        J[2][j] = u[2] * dwt + cz;
    }
    J[0][0] += e.wt; J[1][1] += e.wt; J[2][2] += e.wt;
}

// x = -J^{-1} f by the adjugate; returns false for a singular J
__device__ __forceinline__ bool newton_dir(const double J[3][3], const double* f, double* x)
{
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(fabs(det) > 0.0)) return false;
    const double id = -1.0 / det;
    const double c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const double c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const double c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const double c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    x[0] = (c00 * f[0] + c10 * f[1] + c20 * f[2]) * id;
    x[1] = (c01 * f[0] + c11 * f[1] + c21 * f[2]) * id;
    x[2] = (c02 * f[0] + c12 * f[1] + c22 * f[2]) * id;
    return true;
}

// three floats passed by value (an FP32 copy of u), so they stay in registers
struct F3 {
    float x[3];
};

// FP32 copies of the per-cell constants of the solve, converted once per cell
struct CellF {
    float Es[3], B[3], etat, xi, igh;
};

__device__ __forceinline__ CellF cell_f32(const CellIn& c)
{
    CellF f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        f.Es[i] = d2f_int(c.Es[i]);
        f.B[i] = d2f_int(c.B[i]);
    }
    f.etat = d2f_int(c.etat);
    f.xi = c.xif;
    f.igh = c.ighf;
    return f;
}

// E(u) and dE_i/du_j in FP32 at the FP32 velocity uf (W = Wf, 1/W = iWf)
__device__ __forceinline__ void efield_f32(const CellIn& c, const CellF& cf, const float* uf, float Wf, float iWf,
                                           float* Ef, float dE[3][3])
{
    if (c.emode == 2) {
        DynT<float> dy;
        dyn_coeffs<float>(Wf, cf.etat, cf.xi, dy, true);
        const float s = 1.0f / dy.A[0];
        const float Esu = cf.Es[0] * uf[0] + cf.Es[1] * uf[1] + cf.Es[2] * uf[2];
        const float Bu = cf.B[0] * uf[0] + cf.B[1] * uf[1] + cf.B[2] * uf[2];
        const float ab = dy.A[1] * Esu + dy.A[4] * Bu;
        const float uxEs[3] = {uf[1] * cf.Es[2] - uf[2] * cf.Es[1], uf[2] * cf.Es[0] - uf[0] * cf.Es[2],
                               uf[0] * cf.Es[1] - uf[1] * cf.Es[0]};
        const float uxB[3] = {uf[1] * cf.B[2] - uf[2] * cf.B[1], uf[2] * cf.B[0] - uf[0] * cf.B[2],
                              uf[0] * cf.B[1] - uf[1] * cf.B[0]};
#pragma unroll
        for (int i = 0; i < 3; i++)
            Ef[i] = (cf.etat * cf.Es[i] + ab * uf[i] + dy.A[2] * uxEs[i] + dy.A[3] * cf.B[i] + dy.A[5] * uxB[i]) * s;
        dE_dynamo<float>(dy.A, dy.Ad, Wf, uf, Ef, cf.Es, cf.B, dE);
    } else if (c.emode == 1) {
        const float s = 1.0f / (Wf + cf.etat);
        const float A1 = cf.etat / (1.0f + cf.etat * Wf);
        const float Esu = cf.Es[0] * uf[0] + cf.Es[1] * uf[1] + cf.Es[2] * uf[2];
        const float ae = A1 * Esu;
        Ef[0] = (cf.etat * cf.Es[0] + ae * uf[0] - (uf[1] * cf.B[2] - uf[2] * cf.B[1])) * s;
        Ef[1] = (cf.etat * cf.Es[1] + ae * uf[1] - (uf[2] * cf.B[0] - uf[0] * cf.B[2])) * s;
        Ef[2] = (cf.etat * cf.Es[2] + ae * uf[2] - (uf[0] * cf.B[1] - uf[1] * cf.B[0])) * s;
        const float a2 = A1 * A1 * Esu * iWf;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                dE[i][j] = (-Ef[i] * uf[j] * iWf + A1 * uf[i] * cf.Es[j] - a2 * uf[i] * uf[j] +
                            (i == j ? ae : 0.0f)) * s;
        dE[0][1] -= cf.B[2] * s; dE[0][2] += cf.B[1] * s;
        dE[1][2] -= cf.B[0] * s; dE[1][0] += cf.B[2] * s;
        dE[2][0] -= cf.B[1] * s; dE[2][1] += cf.B[0] * s;
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            Ef[i] = cf.Es[i];
#pragma unroll
            for (int j = 0; j < 3; j++) dE[i][j] = 0.0f;
        }
    }
}

// y = -(J / w_t)^{-1} fs in FP32, J at uf from E, dE, w_t and tau + D - U (= base);
// false when singular
__device__ __forceinline__ bool solve_f32(const CellF& cf, const float* uf, float Wf, float iWf, float uu,
                                          const float* Ef, const float (*dE)[3], float wt, float base, const float* fs,
                                          float* y)
{
    // normalise J by 1/w_t (J = w_t I + ...):
    //   J_ij / w_t = delta_ij + u_i (dw_t/du_j)/w_t + (dE/du_j x B)_i / w_t
    //   (dw_t/du_j)/w_t = ((tau + D - U)/w_t u_j/W - W dU_j/w_t - 2 u_j) / (W^2 - 1/Gamma_hat)
    const float scf = 1.0f / wt;
    const float basef = base * scf;
    const float idenf = 1.0f / (uu + 1.0f - cf.igh);
    float J[3][3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float dU = Ef[0] * dE[0][j] + Ef[1] * dE[1][j] + Ef[2] * dE[2][j];
        const float dw = (basef * uf[j] * iWf - Wf * dU * scf - 2.0f * uf[j]) * idenf;
        const float cx = (dE[1][j] * cf.B[2] - dE[2][j] * cf.B[1]) * scf;
        const float cy = (dE[2][j] * cf.B[0] - dE[0][j] * cf.B[2]) * scf;
        const float cz = (dE[0][j] * cf.B[1] - dE[1][j] * cf.B[0]) * scf;
        J[0][j] = uf[0] * dw + cx;
        J[1][j] = uf[1] * dw + cy;
        J[2][j] = uf[2] * dw + cz;
    }
    J[0][0] += 1.0f; J[1][1] += 1.0f; J[2][2] += 1.0f;
    const float c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const float c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const float c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const float det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(fabsf(det) > 1e-30f)) return false;
    const float id = -scf / det;
    const float c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    const float c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    const float c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    const float c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    const float c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    const float c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    y[0] = (c00 * fs[0] + c10 * fs[1] + c20 * fs[2]) * id;
    y[1] = (c01 * fs[0] + c11 * fs[1] + c21 * fs[2]) * id;
    y[2] = (c02 * fs[0] + c12 * fs[1] + c22 * fs[2]) * id;
    return true;
}

// Newton direction x = -J^{-1} f with J formed and inverted in FP32 (62x the FP64
// rate on GB300).  The root is fixed by the FP64 residual f, so a direction accurate
// to ~1e-6 only turns quadratic convergence into fast linear convergence.  Everything
// J needs is recomputed in FP32 from the FP32 velocity and the per-cell constants,
// except the two FP64 quantities that can cancel (w_t and tau + D - U).  J is
// normalised by w_t and f by the power of two nearest below its scale M (an exact
// rescaling), keeping every float O(1).  Returns false when the FP32 system is
// singular or the direction is not finite (the caller then uses the FP64 Jacobian).
__device__ __forceinline__ bool newton_dir_f32(const CellIn& c, const CellF& cf, const double* u, const Eval& e,
                                               double* x, bool has_uin, const F3& uin)
{
    float uf[3];
#pragma unroll
    for (int i = 0; i < 3; i++) uf[i] = has_uin ? uin.x[i] : d2f_int(u[i]);
    const float uu = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
    const float Wf = sqrtf(1.0f + uu), iWf = 1.0f / Wf;
    float Ef[3], dE[3][3];
    efield_f32(c, cf, uf, Wf, iWf, Ef, dE);
    // f scaled by 2^-k with 2^k <= M < 2^(k+1): the exponent field of M, read as an integer
    const int ek = (int)(mag_hi(e.M) >> 20);
    const bool scale = ek >= 1 && ek <= 2045;
    const double down = scale ? __hiloint2double((2046 - ek) << 20, 0) : 1.0;
    const double up = scale ? __hiloint2double(ek << 20, 0) : 1.0;
    const float fs[3] = {d2f_int(e.f[0] * down), d2f_int(e.f[1] * down), d2f_int(e.f[2] * down)};
    float y[3];
    if (!solve_f32(cf, uf, Wf, iWf, uu, Ef, dE, d2f_int(e.wt), d2f_int(c.tD - e.U), fs, y)) return false;
    // (J / w_t) y = -(f 2^-k) / w_t  ->  x = 2^k y
    x[0] = up * f2d_int(y[0]);
    x[1] = up * f2d_int(y[1]);
    x[2] = up * f2d_int(y[2]);
    return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

// One Newton step done wholly in FP32 (residual, Jacobian and solve) from the start u:
// the residual of a start within ~1e-6 of the root is then accurate to a few per cent,
// enough to bring the start to FP32 accuracy (~1e-7) before the FP64 iteration, which
// then needs one FP64 evaluation fewer.  u is moved only when the step is finite and
// within the step bound; the FP64 iteration fixes the root as before.  uin: the FP32
// value of u when the caller has it (has_uin; else converted here); when u moves, uout
// gets the FP32 sum, within an FP32 rounding of the new u (all the next FP32 direction
// needs).  Returns whether u moved.
__device__ __forceinline__ bool newton_step_f32(const CellIn& c, const CellF& cf, double* u, bool has_uin,
                                                const F3& uin, F3& uout)
{
    float uf[3];
#pragma unroll
    for (int i = 0; i < 3; i++) uf[i] = has_uin ? uin.x[i] : d2f_int(u[i]);
    const float uu = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
    const float Wf = sqrtf(1.0f + uu), iWf = 1.0f / Wf;
    float Ef[3], dE[3][3];
    efield_f32(c, cf, uf, Wf, iWf, Ef, dE);
    const float U = 0.5f * (Ef[0] * Ef[0] + Ef[1] * Ef[1] + Ef[2] * Ef[2] + cf.B[0] * cf.B[0] + cf.B[1] * cf.B[1] +
                            cf.B[2] * cf.B[2]);
    const float Sf[3] = {d2f_int(c.S[0]), d2f_int(c.S[1]), d2f_int(c.S[2])};
    const float Df = d2f_int(c.D);
    const float base = d2f_int(c.tD) - U;
    const float wt = (Wf * base - Df * cf.igh) / (uu + 1.0f - cf.igh);
    const float x0 = Ef[1] * cf.B[2] - Ef[2] * cf.B[1];
    const float x1 = Ef[2] * cf.B[0] - Ef[0] * cf.B[2];
    const float x2 = Ef[0] * cf.B[1] - Ef[1] * cf.B[0];
    // f / M with M the momentum scale (as in evaluate)
    const float M = fmaxf(fmaxf(fmaxf(fabsf(Sf[0]), fabsf(Sf[1])), fmaxf(fabsf(Sf[2]), fabsf(x0))),
                          fmaxf(fmaxf(fabsf(x1), fabsf(x2)),
                                fmaxf(fabsf(wt * uf[0]), fmaxf(fabsf(wt * uf[1]), fabsf(wt * uf[2])))));
    if (!(wt > 0.0f) || !(M > 0.0f) || !(M < 1e30f)) return false;
    const float iM = 1.0f / M;
    const float fs[3] = {(wt * uf[0] - Sf[0] + x0) * iM, (wt * uf[1] - Sf[1] + x1) * iM,
                         (wt * uf[2] - Sf[2] + x2) * iM};
    float y[3];
    if (!solve_f32(cf, uf, Wf, iWf, uu, Ef, dE, wt, base, fs, y)) return false;
    const float dx[3] = {y[0] * M, y[1] * M, y[2] * M};
    const float nx2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    if (!(nx2 <= 1e4f * fmaxf(1.0f, uu))) return false;   // also rejects NaN
#pragma unroll
    for (int i = 0; i < 3; i++) {
        u[i] += f2d_int(dx[i]);
        uout.x[i] = uf[i] + dx[i];
    }
    return true;
}

// ---------------------------------------------------------------------------
// double-word residual (dword.cuh): the Newton corrections of the implicit solve are
// formed on the FP32 pipe from a residual accurate to ~1e-14; only the final residual,
// which accepts the root, is evaluated in FP64
// ---------------------------------------------------------------------------

// x as a double-word pair, on the integer pipe: hi = d2f_int(x), and lo = x - hi
// (exact in binary64) rounded to binary32.  With L the 29 significand bits that hi
// drops and r = L, or L - 2^29 where hi rounded up, |x| - |hi| = r 2^(e - 1075) for
// the biased exponent e.  r (|r| <= 2^28) becomes a float as rh 2^14 + rl, each half
// converted exactly by the 1.5 2^23 bias (rh < 2^14 and rl < 2^14 in magnitude), with
// one rounding in the final fma.  Outside binary32's normal range, or where lo would
// fall below it (|x| < 2^-74), lo is 0: the pair is then only binary32-accurate, which
// the FP64 residual that accepts the root detects.
__device__ __forceinline__ dw dw_of(double x)
{
    const unsigned whi = (unsigned)__double2hiint(x), wlo = (unsigned)__double2loint(x);
    const unsigned e = (whi >> 20) & 0x7ffu;
    const float h = d2f_int(x);
    if (e - 949u > 201u) return {h, 0.0f};   // e outside [949, 1150]
    const int r = (int)(wlo & 0x1fffffffu) - (int)((wlo >> 28) & 1u) * (1 << 29);
    const float fh = __fsub_rn(__int_as_float(0x4B400000 + (r >> 14)), 12582912.0f);
    const float fl = __fsub_rn(__int_as_float(0x4B400000 + (r & 0x3fff)), 12582912.0f);
    const float sc = __uint_as_float((e - 948u) << 23);   // 2^(e - 1075)
    const float l = fmaf(fh, __fmul_rn(16384.0f, sc), __fmul_rn(fl, sc));
    return {h, (whi >> 31) ? -l : l};
}

__device__ __forceinline__ double dw_to_double(dw x) { return f2d_int(x.hi) + f2d_int(x.lo); }

__device__ __forceinline__ dw dw_dot3(const dw* a, const dw* b)
{
    return dw_add(dw_add(dw_mul(a[0], b[0]), dw_mul(a[1], b[1])), dw_mul(a[2], b[2]));
}

// (a x b)_i = a_j b_k - a_k b_j
__device__ __forceinline__ dw dw_cross(const dw* a, const dw* b, int i)
{
    const int j = (i + 1) % 3, k = (i + 2) % 3;
    return dw_sub(dw_mul(a[j], b[k]), dw_mul(a[k], b[j]));
}

// The residual f = w_t u - S + E x B of evaluate() in double-word arithmetic, for the
// resistive and E-fixed forms of E(u) (emode 1 and 0).  The per-cell constants are
// split from their FP64 values on the integer pipe.  Outputs in binary32: f (each
// accurate to ~1e-14 of the momentum scale), w_t, tau + D - U and the scale M.
struct EvalDW {
    float f[3], wt, base, M;
};

// W, E(u) and w_t of the last double-word evaluation, kept when the residual there
// accepts the root (double-word acceptance)
struct DwRoot {
    dw W, wt, E[3];
};

template <bool KEEP = false>
__device__ __forceinline__ void evaluate_dw(const CellIn& c, const dw* u, EvalDW& o, DwRoot* r = nullptr)
{
    dw S[3], B[3], E[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        S[i] = dw_of(c.S[i]);
        B[i] = dw_of(c.B[i]);
    }
    const dw Wsq = dw_add_f(dw_add(dw_add(dw_sqr(u[0]), dw_sqr(u[1])), dw_sqr(u[2])), 1.0f);
    const dw W = dw_sqrt(Wsq);
    if (c.emode == 1) {
        // A_0 E = eta_t E* + A_1 (E*.u) u - u x B, A_0 = W + eta_t, A_1 = eta_t/(1 + eta_t W)
        const dw et = dw_of(c.etat);
        dw Es[3];
#pragma unroll
        for (int i = 0; i < 3; i++) Es[i] = dw_of(c.Es[i]);
        const dw iWe = dw_rcp(dw_add(W, et));
        const dw A1 = dw_mul(et, dw_rcp(dw_add_f(dw_mul(et, W), 1.0f)));
        const dw ae = dw_mul(A1, dw_dot3(Es, u));
#pragma unroll
        for (int i = 0; i < 3; i++)
            E[i] = dw_mul(dw_sub(dw_add(dw_of(c.etEs[i]), dw_mul(ae, u[i])), dw_cross(u, B, i)), iWe);
    } else {
#pragma unroll
        for (int i = 0; i < 3; i++) E[i] = dw_of(c.Es[i]);
    }
    // U = |E|^2/2 + |B|^2/2;  w_t = (W (tau + D - U) - D/Gamma_hat) / (W^2 - 1/Gamma_hat)
    const dw U = dw_add(dw_scale(dw_dot3(E, E), 0.5f), dw_of(c.B2h));
    const dw base = dw_sub(dw_of(c.tD), U);
    const dw wt = dw_mul(dw_sub(dw_mul(W, base), dw_of(c.Digh)), dw_rcp(dw_sub(Wsq, dw_of(c.igh))));
    float M = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const dw x = dw_cross(E, B, i);
        const dw w = dw_mul(wt, u[i]);
        o.f[i] = dw_add(dw_sub(w, S[i]), x).hi;
        M = fmaxf(M, fmaxf(fabsf(S[i].hi), fmaxf(fabsf(x.hi), fabsf(w.hi))));
    }
    o.wt = wt.hi;
    o.base = base.hi;
    o.M = M;
    if (KEEP) {
        r->W = W;
        r->wt = wt;
#pragma unroll
        for (int i = 0; i < 3; i++) r->E[i] = E[i];
    }
}

// Newton corrections from the double-word residual with the FP32 Jacobian (the
// direction of newton_dir_f32, here at the double-word velocity), at most `nit`
// evaluations.  It stops once |f| <= tol M / 4 in double-word arithmetic, or after a
// step |dx|^2 <= tol max(|u|^2, 1) / 100: the FP32 Jacobian contracts the error by
// ~1e-6 per step and the quadratic term is ~|dx|^2, so the residual after such a step
// is already below the tolerance and the FP64 residual can accept it directly.  Steps
// are taken only when finite and within the step bound; u (FP64) receives the result
// only if it is finite.
//
// ACC (double-word acceptance, for tolerances of 1e-11 and above): the double-word
// residual itself accepts the root.  It is accurate to ~1e-14 of the momentum scale,
// a few hundred times below tol M / 4 there, so |f| <= tol M / 4 in double-word
// arithmetic bounds the exact residual by the tolerance.  The small-step exit is then
// skipped (the next evaluation decides), and on acceptance u, W, 1/W, w_t and E(u)
// are written to e from the double-word values; the return value says whether that
// happened (else the FP64 residual decides, as without ACC).
constexpr int kDwEvals = 4;   // most double-word residual evaluations per solve
constexpr unsigned kHi1e10 = 0x4202A05Fu;   // high word of 1e10 (the bound on W)

template <bool ACC>
__device__ __forceinline__ bool newton_refine_dw(const CellIn& c, const CellF& cf, double* u, float tol, int nit,
                                                 Eval* e)
{
    dw ud[3];
#pragma unroll
    for (int i = 0; i < 3; i++) ud[i] = dw_of(u[i]);
    bool moved = false;
    for (int k = 0; k < nit; k++) {
        EvalDW ed;
        DwRoot rt;
        evaluate_dw<ACC>(c, ud, ed, &rt);
        if (!(ed.M > 0.0f) || !(ed.M < 1e30f) || !(ed.wt > 0.0f)) break;
        const float fm = fmaxf(fabsf(ed.f[0]), fmaxf(fabsf(ed.f[1]), fabsf(ed.f[2])));
        if (fm <= 0.25f * tol * ed.M) {   // also false for NaN
            if (ACC && rt.W.hi < 1e10f) {
                const dw iW = dw_rcp(rt.W);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    u[i] = dw_to_double(ud[i]);
                    e->E[i] = dw_to_double(rt.E[i]);
                }
                e->W = dw_to_double(rt.W);
                e->iW = dw_to_double(iW);
                e->wt = dw_to_double(rt.wt);
                return true;
            }
            break;
        }
        const float uf[3] = {ud[0].hi, ud[1].hi, ud[2].hi};
        const float uu = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
        const float Wf = sqrtf(1.0f + uu), iWf = 1.0f / Wf;
        float Ef[3], dE[3][3];
        efield_f32(c, cf, uf, Wf, iWf, Ef, dE);
        const float iM = 1.0f / ed.M;
        const float fs[3] = {ed.f[0] * iM, ed.f[1] * iM, ed.f[2] * iM};
        float y[3];
        if (!solve_f32(cf, uf, Wf, iWf, uu, Ef, dE, ed.wt, ed.base, fs, y)) break;
        const float dx[3] = {y[0] * ed.M, y[1] * ed.M, y[2] * ed.M};
        const float nx2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        if (!(nx2 <= 1e4f * fmaxf(1.0f, uu))) break;   // also rejects NaN
#pragma unroll
        for (int i = 0; i < 3; i++) ud[i] = dw_add_f(ud[i], dx[i]);
        moved = true;
        if (!ACC && nx2 <= 0.01f * tol * fmaxf(1.0f, uu)) break;
    }
    if (moved) {
        const double v[3] = {dw_to_double(ud[0]), dw_to_double(ud[1]), dw_to_double(ud[2])};
        if (finite_int(v[0]) && finite_int(v[1]) && finite_int(v[2])) {
            u[0] = v[0];
            u[1] = v[1];
            u[2] = v[2];
        }
    }
    return false;
}

// Globally convergent Newton (backtracking on |f|^2 with the Armijo condition and a
// bounded step).  u: in = initial guess, out = solution.  Converged when |f| is at
// `tol` against its own momentum scale M, or when the step no longer moves u.
// Returns iterations, or -1.  uin: the FP32 value of the start when the caller has it
// (has_uin; the start is then exactly that value).  ACC: double-word acceptance (the
// mixed-precision path, whose tolerance is at least 1e-11; see newton_refine_dw).
template <bool ACC = false>
__device__ __forceinline__ int newton_solve(const CellIn& c, double* u, Eval& e, int kmax, double tol, float tolf,
                                            bool has_uin, const F3& uin)
{
    const CellF cf = cell_f32(c);
    // the FP32 first step saves an FP64 evaluation only when the tolerance lies below
    // what one FP64 iteration reaches from a start ~1e-6 off (~1e-12): the FP64 path's
    // 1e-13, not the mixed path's 1e-10
    F3 uf1 = uin;   // FP32 value of u at the first direction (when has1)
    bool has1 = has_uin;
    if (c.emode != 2) {
        // Newton corrections from the double-word residual; the FP64 residual below
        // then accepts the root (or, with ACC, the double-word one already did), or the
        // FP64 iteration continues from there
        if (newton_refine_dw<ACC>(c, cf, u, tolf, kDwEvals, &e)) return 0;
        has1 = false;
    } else if (tol < 1e-11) {
        F3 un;
        if (newton_step_f32(c, cf, u, has_uin, uin, un)) {
            uf1 = un;
            has1 = true;
        }
    }
    evaluate(c, u, e);
    if (e.fm <= tol * e.M) {
        if (!pos_int(e.wt) || !mag_below_int(e.W, kHi1e10)) return -1;
        return 0;
    }
    for (int it = 1; it <= kmax; it++) {
        double dx[3];
        // FP32 directions first; the FP64 Jacobian takes over if they have not
        // converged within 10 iterations or fail
        if (it > 10 || !newton_dir_f32(c, cf, u, e, dx, it == 1 && has1, uf1)) {
            double J[3][3];
            jacobian(c, u, e, J);
            if (!newton_dir(J, e.f, dx)) return -1;
        }
        // step bound |dx| <= 100 max(|u|, 1), compared in squares
        const double nu2 = fmax(1.0, u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double nx2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        if (nx2 > 1e4 * nu2) {
            const double s = sqrt(1e4 * nu2 / nx2);
            dx[0] *= s; dx[1] *= s; dx[2] *= s;
        }
        // slope of |f|^2 along the Newton direction is -2|f|^2 (|f|^2 is formed here,
        // not in evaluate: a residual accepted at once never needs it)
        const double g0 = fnorm2(e);
        double lam = 1.0, ut[3];
        Eval et;
        for (int ls = 0; ls < 30; ls++) {
            ut[0] = u[0] + lam * dx[0]; ut[1] = u[1] + lam * dx[1]; ut[2] = u[2] + lam * dx[2];
            evaluate(c, ut, et);
            const double gt = fnorm2(et);
            if (gt <= g0 * (1.0 - 2e-4 * lam) || !(g0 > 0.0)) break;
            double lq = g0 * lam * lam / (gt - g0 + 2.0 * g0 * lam);
            if (!(lq == lq)) lq = 0.5 * lam;
            lam = fmin(fmax(lq, 0.1 * lam), 0.5 * lam);
        }
        const double step = lam * from_hi(max(mag_hi(dx[0]), max(mag_hi(dx[1]), mag_hi(dx[2]))));
        u[0] = ut[0]; u[1] = ut[1]; u[2] = ut[2];
        e = et;
        const double umax = from_hi(max(mag_hi(u[0]), max(mag_hi(u[1]), mag_hi(u[2]))));
        if (e.fm <= tol * e.M || step <= 1e-15 * umax) {
            if (!pos_int(e.wt) || !mag_below_int(e.W, kHi1e10)) return -1;
            return it;
        }
    }
    return -1;
}

}  // namespace grmhd
