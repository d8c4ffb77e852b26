// sweep_bodies.cuh -- device code of one SIMPLE-TS time step
// (K. S. Shterev, arXiv:1802.04243, Sections 3.1 and 3.2) shared by the
// per-phase kernels and the persistent step kernel of batches
// (phase_kernels.cuh, compiled per arithmetic in phase_*.cu and step_*.cu)
// and by the support kernels of sweep_kernels.cu: the equation bodies of every
// phase, templated on the arithmetic, the residual reduction and the
// tile-list walk.  Every kernel compiles these same bodies, so a position's
// arithmetic is the same whichever kernel runs it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "stg_common.cuh"

namespace stg {
namespace {

constexpr int BX = 32, BY = 8;

struct Ix {
    int P;
    __device__ __forceinline__ int operator()(int i, int j) const { return (j + G) * P + (i + G); }
};

template <typename R>
__device__ __forceinline__ R at(const R *a, int i) { return a[i + G]; }

// vel > 0 from the bit pattern: a positive double (float) is a positive
// 64-bit (32-bit) integer, so the test runs on the integer pipe instead of
// GB300's narrow FP64 pipe.  (NaN inputs may take either branch.)
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return __float_as_int(x) > 0; }
__device__ __forceinline__ bool positive(df64 x) { return x.hi > 0.0f; }    // normalised: lo is 0 when hi is

// x < 0, the same test as positive(-x) without forming -x (-0 is not below
// zero): sign bit set and a nonzero rest.
__device__ __forceinline__ bool below_zero(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) != 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool below_zero(float x)
{
    const unsigned b = __float_as_uint(x);
    return (b >> 31) != 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool below_zero(df64 x) { return positive(-x); }

// x != 0 (either sign of zero counts as zero), from the bits.
__device__ __forceinline__ bool nonzero(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ bool nonzero(float x) { return (__float_as_uint(x) << 1) != 0; }
__device__ __forceinline__ bool nonzero(df64 x) { return x.hi != 0.0f; }

// max(0, -x), the same bits as pos(-x): the sign test reads the sign bit and
// the FP64 negation flips it on the integer pipe.
__device__ __forceinline__ bool negative(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool negative(float x) { return __float_as_int(x) < 0; }
__device__ __forceinline__ bool negative(df64 x) { return positive(-x); }
__device__ __forceinline__ double flip_sign(double x)
{
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000u, __double2loint(x));
}
__device__ __forceinline__ float flip_sign(float x) { return -x; }
__device__ __forceinline__ df64 flip_sign(df64 x) { return -x; }
template <typename R>
__device__ __forceinline__ R neg_part(R x) { return negative(x) ? flip_sign(x) : R(0); }

// ---------------------------------------------------------------- limiter

__device__ __forceinline__ float recip(float a);
__device__ __forceinline__ double recip(double a);

// Van Leer psi(r) = (r + |r|)/(1 + r) for r = num/den, i.e. 2 num/(num + den)
// when num and den are nonzero with one sign, else 0 (a zero denominator
// falls back to first order).  Its half, num/(num + den), is what the
// corrections below use (the factor 2 is folded into their weights; scaling
// by a power of two is exact).  The sign test reads the sign bits, so it
// runs on the integer pipe; the quotient uses the sweep's reciprocal.
template <typename R>
__device__ __forceinline__ R van_leer_half(R num, R den)
{
    const bool same = (positive(num) && positive(den)) || (below_zero(num) && below_zero(den));
    return same ? num * recip(num + den) : R(0);
}

// Eq. pl15_2: correction at the face between nodes 2 and 3 for flow towards
// node 3 (up) and towards node 2 (dn), with d1..d4 the sizes of the four
// nodes: psi = w2 VanLeer((d2 + d3)(f2 - f1), (d1 + d2)(f3 - f2)) and its
// mirror, w2 = d2/(d2 + d3), w3 = d3/(d2 + d3).  Van Leer's quotient is
// unchanged when both arguments are halved, so the sums of two sizes enter
// as the centre distances c12 = (d1 + d2)/2, c23, c34 of the axis tables, and
// w2 VanLeer = (2 w2) VanLeer/2 with 2 w2 tabulated (the same bits: every
// rescaling is by a power of two).
template <typename R>
__device__ __forceinline__ R psi_s_up(R f1, R f2, R f3, R c12, R c23, R w2x2)
{
    return w2x2 * van_leer_half(c23 * (f2 - f1), c12 * (f3 - f2));
}
template <typename R>
__device__ __forceinline__ R psi_s_dn(R f2, R f3, R f4, R c23, R c34, R w3x2)
{
    return -(w3x2 * van_leer_half(c23 * (f4 - f3), c34 * (f3 - f2)));
}
template <typename R>
__device__ __forceinline__ R psi_surface(R f1, R f2, R f3, R f4, R c12, R c23, R c34, R w2x2, R w3x2, R vel)
{
    return positive(vel) ? psi_s_up(f1, f2, f3, c12, c23, w2x2) : psi_s_dn(f2, f3, f4, c23, c34, w3x2);
}

// Eq. pl15_1: face midway between nodes 2 and 3; d1..d3 the node distances;
// psi = +-0.5 VanLeer(...).
template <typename R>
__device__ __forceinline__ R psi_centre(R f1, R f2, R f3, R f4, R d1, R d2, R d3, R vel)
{
    if (positive(vel))
        return van_leer_half(d2 * (f2 - f1), d1 * (f3 - f2));
    return flip_sign(van_leer_half(d2 * (f4 - f3), d3 * (f3 - f2)));
}

template <typename R>
__device__ __forceinline__ R upwind(R a, R b, R vel) { return positive(vel) ? a : b; }
template <typename R>
__device__ __forceinline__ R pos(R x) { return positive(x) ? x : R(0); }


// Value of node m seen from node a: reflected about the stored wall value when
// the flag of m carries `wall_bit`.
template <typename R, bool WALLS = true>
__device__ __forceinline__ R seen(const R *f, const uint16_t *flag, int a, int m, uint32_t wall_bit)
{
    R fm = f[m];
    if constexpr (!WALLS)
        return fm;                 // caller knows no wall is in reach
    else
        return (flag[m] & wall_bit) ? R(2) * fm - f[a] : fm;
}


// Value of node m seen from node a when m may lie across a wall or obstacle
// (the flag of m carries wall_bit): reflected about the value at the wall
// surface, phi_s = (h phi_w + s phi_a)/(h + s), Eqs. pl38, pl39 with the
// normal derivative (phi_a - phi_s)/h; h is half the reader's size normal to
// the wall, s = coef / rho_local with rho_local the mean of rho[r0] and
// rho[r1] (the reader's cell, or the two cells of its u or v control volume).
// coef = 0: the no-slip / isothermal reflection 2 phi_w - phi_a.
template <typename R, bool WALLS = true>
__device__ __forceinline__ R seen_s(const R *f, const uint16_t *flag, int a, int m, uint32_t wall_bit, R coef,
                                    R size, const R *rho, int r0, int r1)
{
    const R fm = f[m];
    if constexpr (!WALLS) {
        return fm;
    } else {
        if (!(flag[m] & wall_bit)) return fm;
        const R fa = f[a];
        if (!positive(coef)) return R(2) * fm - fa;
        const R sl = coef * recip(R(0.5) * (rho[r0] + rho[r1]));
        const R h = R(0.5) * size;
        return R(2) * ((h * fm + sl * fa) * recip(h + sl)) - fa;
    }
}

// Gamma at the corner (x^f_i, y^f_j): bilinear in the four cell centres.
template <typename R>
__device__ __forceinline__ R gamma_corner(const GeoT<R> &g, const R *gam, int c, int i, int j)
{
    const int P = g.pitch;
    R lo = at(g.x.wlo, i) * gam[c - P - 1] + at(g.x.whi, i) * gam[c - P];
    R hi = at(g.x.wlo, i) * gam[c - 1] + at(g.x.whi, i) * gam[c];
    return at(g.y.wlo, j) * lo + at(g.y.whi, j) * hi;
}

// 2 C^T1_f times the length d of a face at index q of an axis: tabulated in
// FP64 (a load instead of an FP64 multiply), formed in the branch that uses
// it by the FP32 and double-float sweeps from ct1f2 = 2 C^T1_f (forming both
// faces' factors up front made the double-float face kernel 15 % slower).
template <typename R>
__device__ __forceinline__ R face_ct2(const AxisT<R> &ax, int q, R ct1f2, R d)
{
    if constexpr (std::is_same<R, double>::value)
        return at(ax.ct2d, q);
    else
        return ct1f2 * d;
}

// Volume of cell (i,j) per unit time, dx_i dy_j / dt: the factor of the
// transient terms of Eqs. pl30 and pl24 once those equations are divided by
// dt (as the momentum equations Eqs. pl14-pl16 are written).  FP64 takes
// dy_j / dt from the axis table.
template <typename R>
__device__ __forceinline__ R vol_per_dt(const GeoT<R> &g, const CoefT<R> &k, int j, R dxi, R dyj)
{
    if constexpr (std::is_same<R, double>::value)
        return dxi * at(g.y.dt1, j);
    else
        return dxi * (dyj * (R(2) * k.hrdt));
}

// ------------------------------------------------------ residual reduction

// Ordered key of |x|: the bits of an FP64 value without its sign, ordered like
// |x| as unsigned integers, NaN above infinity.  The sign is cleared by a
// 32-bit AND on the high word (inline PTX): written as a 64-bit mask, the
// compiler had turned it into an FP64 absolute value, one instruction on
// GB300's narrow FP64 pipe per residual.
__device__ __forceinline__ unsigned long long ordered_bits(double x)
{
    unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    asm("and.b32 %0, %0, 0x7fffffff;" : "+r"(hi));
    return ((unsigned long long)hi << 32) | lo;
}

// FP32 <-> FP64 conversions on the integer pipe.  On GB300 the F2F
// instructions issue on the FP64 pipe (1/64 of the FP32 rate); the mixed path
// converts every value it moves between the two precisions, so it assembles
// the IEEE bit patterns itself.
// widen: exact FP32 -> FP64 (FP32 subnormals become zero).
__device__ __forceinline__ double widen(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    unsigned hi = sgn | ((e + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (e == 0u) {
        hi = sgn;
        lo = 0u;
    } else if (e == 0xFFu) {
        hi = sgn | 0x7FF00000u | (m >> 3);
    }
    return __hiloint2double((int)hi, (int)lo);
}

// narrow: FP64 -> FP32 rounded to nearest (ties away from zero); magnitudes
// below the FP32 normal range become zero, above it infinity; NaN stays NaN.
__device__ __forceinline__ float narrow(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned sgn = hi & 0x80000000u, e64 = (hi >> 20) & 0x7FFu;
    const int e = (int)e64 - 896;
    const unsigned mag = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    unsigned bits;
    if (e64 == 0x7FFu)
        bits = 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
    else if (e <= 0)
        bits = 0u;
    else if (e >= 255)
        bits = 0x7F800000u;
    else
        bits = (((unsigned)e << 23) | mag) + ((lo >> 28) & 1u);
    return __uint_as_float(sgn | bits);
}

__device__ __forceinline__ void block_max2(unsigned long long a, unsigned long long b,
                                           unsigned long long *da, unsigned long long *db)
{
    __shared__ unsigned long long sa[32], sb[32];
    for (int o = 16; o > 0; o >>= 1) {
        a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
    if (lane == 0) { sa[warp] = a; sb[warp] = b; }
    __syncthreads();
    if (warp == 0) {
        a = lane < nw ? sa[lane] : 0ull;
        b = lane < nw ? sb[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            if (a) atomicMax(da, a);
            if (b) atomicMax(db, b);
        }
    }
    __syncthreads();       // the shared slots are reused by the block's next call
}

// 1/a.  FP64: from the FP32 reciprocal r of a (relative error e = 1 - a r
// below about 2^-23), one third-order step of the geometric series
// 1/a = r / (1 - e) = r (1 + e + e^2 + ...), r <- r + r (e + e^2), three
// fused multiply-adds; the truncation leaves about e^3 < 2^-69, so the result
// is within one ulp of 1/a.  It replaces the longer IEEE division sequence on
// GB300's slow FP64 pipe.  Magnitudes outside [2^-100, 2^100] fall back to the
// IEEE division.  FP32: the IEEE division.
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }
__device__ __forceinline__ double recip(double a)
{
    const unsigned ex = ((unsigned)__double2hiint(a) >> 20) & 0x7FFu;
    if (ex < 1023u - 100u || ex > 1023u + 100u)
        return 1.0 / a;
    const double r = widen(1.0f / narrow(a));
    const double e = fma(-a, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// Residual key |d| of a difference held in the compute precision (a
// double-float difference is keyed by its leading float).
__device__ __forceinline__ unsigned long long res_key(double d) { return ordered_bits(d); }
__device__ __forceinline__ unsigned long long res_key(df64 d) { return ordered_bits(widen(d.hi)); }

// d/2 of index i: from the half-size table in FP64 (a load instead of an
// FP64 multiply); the FP32 and double-float sweeps, bound by latency rather
// than by arithmetic, multiply (the same value: halving is exact).
template <typename R>
__device__ __forceinline__ R half_size(const AxisT<R> &ax, int i, R d)
{
    if constexpr (std::is_same<R, double>::value)
        return ax.hd[i + G];
    else
        return R(0.5) * d;
}

// sqrt(T) for Gamma with omega = 1/2: from the FP32 reciprocal square root y
// of T, s = T y and two Newton-Raphson steps for s^2 = T,
// s <- s + (T - s^2) (y/2), each a fused multiply-add for the residual and
// one for the update.  The relative error falls from about 2^-22 to about
// 2^-65, so the result is within one ulp of the correctly rounded root, in
// five FP64 instructions.  Magnitudes outside [2^-100, 2^100] use sqrt.
__device__ __forceinline__ double root(double T)
{
    const unsigned ex = ((unsigned)__double2hiint(T) >> 20) & 0x7FFu;
    if (ex < 1023u - 100u || ex > 1023u + 100u)
        return sqrt(T);
    const float y = rsqrtf(narrow(T));
    const double h = widen(0.5f * y);
    double s = T * widen(y);
    s = fma(fma(-s, s, T), h, s);
    return fma(fma(-s, s, T), h, s);
}

// Gamma = T^omega (power-law transport coefficients): the square root for
// omega = 1/2, the general power otherwise (double-float: through FP64).
// (omega == 1/2 is tested on the bits, keeping the comparison off the FP64 pipe)
__device__ __forceinline__ bool is_half(double omega) { return __double_as_longlong(omega) == 0x3FE0000000000000LL; }
__device__ __forceinline__ double gamma_of(double T, double omega) { return is_half(omega) ? root(T) : pow(T, omega); }
__device__ __forceinline__ df64 gamma_of(df64 T, df64 omega)
{
    if (omega.hi == 0.5f && omega.lo == 0.0f) return sqrt(T);
    return dfl::split_dev(pow(dfl::join(T), dfl::join(omega)));
}

// T conductance of the face between a node of size da and one of size db
// (Eq. pl32): c_area Gamma_f / (0.5 (da + db)) with the distance-weighted
// harmonic mean Gamma_f = (da + db) ga gb / (da gb + db ga) of Eq. pl33,
// i.e. 2 c_area ga gb / (da gb + db ga).  c2_area = 2 C^T1_f times the face
// area (the caller doubles C^T1_f once for both faces; doubling is exact).
template <typename R>
__device__ __forceinline__ R conductance(R ga, R gb, R da, R db, R c2_area)
{
    return c2_area * (ga * gb) * recip(fma(da, gb, db * ga));
}

// ------------------------------------------------------- face densities

// The TVD limiters of position (i,j) (WorkT::psTx ... psVxD), each from the
// level's own fields and written as 0 where the flag says the four stencil
// nodes are not all unknowns (so no wall value enters a limiter).
template <typename R>
__device__ __forceinline__ void face_limiters(const GeoT<R> &g, const R *__restrict__ u, const R *__restrict__ v,
                                              const R *__restrict__ T, const WorkT<R> &w, int c, int i, int j)
{
    const int P = g.pitch;
    const uint16_t f = g.flag[c];
    const R zero = R(0);
    // T on the x face i and the y face j (Eq. pl15_2)
    w.psTx[c] = (f & F_TCX) ? psi_surface(T[c - 2], T[c - 1], T[c], T[c + 1], at(g.x.dc, i - 1), at(g.x.dc, i),
                                          at(g.x.dc, i + 1), at(g.x.whi2, i), at(g.x.wlo2, i), u[c])
                            : zero;
    w.psTy[c] = (f & F_TCY) ? psi_surface(T[c - 2 * P], T[c - P], T[c], T[c + P], at(g.y.dc, j - 1), at(g.y.dc, j),
                                          at(g.y.dc, j + 1), at(g.y.whi2, j), at(g.y.wlo2, j), v[c])
                            : zero;
    // u node (i,j): x face of its control volume at the centre of cell i-1
    // (Eq. pl15_1, velocity the mean of the two u nodes), and the y face
    // between u nodes (i,j-1) and (i,j) (Eq. pl15_2, both flow directions)
    // (only the sign of the mean velocity selects the branch: the sum has it)
    w.psUx[c] = (f & F_TUX) ? psi_centre(u[c - 2], u[c - 1], u[c], u[c + 1], at(g.x.d, i - 2), at(g.x.d, i - 1),
                                         at(g.x.d, i), u[c - 1] + u[c])
                            : zero;
    // (a branch is evaluated only if one of the two v faces that select it,
    // v(i-1,j) and v(i,j), points its way)
    {
        const bool t = (f & F_TUY) != 0, p0 = positive(v[c - 1]), p1 = positive(v[c]);
        w.psUyU[c] = (t && (p0 || p1)) ? psi_s_up(u[c - 2 * P], u[c - P], u[c], at(g.y.dc, j - 1), at(g.y.dc, j),
                                                  at(g.y.whi2, j))
                                       : zero;
        w.psUyD[c] = (t && !(p0 && p1)) ? psi_s_dn(u[c - P], u[c], u[c + P], at(g.y.dc, j), at(g.y.dc, j + 1),
                                                   at(g.y.wlo2, j))
                                        : zero;
    }
    // v node (i,j): the mirror image
    w.psVy[c] = (f & F_TVY) ? psi_centre(v[c - 2 * P], v[c - P], v[c], v[c + P], at(g.y.d, j - 2), at(g.y.d, j - 1),
                                         at(g.y.d, j), v[c - P] + v[c])
                            : zero;
    {
        const bool t = (f & F_TVX) != 0, p0 = positive(u[c - P]), p1 = positive(u[c]);
        w.psVxU[c] = (t && (p0 || p1)) ? psi_s_up(v[c - 2], v[c - 1], v[c], at(g.x.dc, i - 1), at(g.x.dc, i),
                                                  at(g.x.whi2, i))
                                       : zero;
        w.psVxD[c] = (t && !(p0 && p1)) ? psi_s_dn(v[c - 1], v[c], v[c + 1], at(g.x.dc, i), at(g.x.dc, i + 1),
                                                   at(g.x.wlo2, i))
                                        : zero;
    }
}

// Per-position face quantities of one state level, stored for the kernels
// that follow: rho^u dy at u face (i,j) and rho^v dx at v face (i,j) (the
// face densities of Eqs. pl10, pl11 -- the upwind value plus psi_s times the
// difference across the face -- times the face area), the mass fluxes
// through them (Eqs. pl8, pl9), the T conductances of the x
// and y faces (Eq. pl32 with the harmonic mean Eq. pl33), B Gamma at the
// corner (x^f_i, y^f_j), and the normal-stress conductances B Gamma dy/dx,
// B Gamma dx/dy of cell (i,j).  Each is used by two to four neighbours in the
// assembly, which would otherwise recompute it each time.
// With `limiters` (TVD only) it also evaluates the Van Leer limiters of the
// level once per face for the temperature and momentum equations, which
// would otherwise be evaluated by both control volumes sharing the face.
template <typename R, bool TVD>
__device__ __forceinline__ void face_densities_body(const GeoT<R> &g, const CoefT<R> &k, const R *__restrict__ u,
                                                    const R *__restrict__ v, const R *__restrict__ rho,
                                                    const R *__restrict__ gam, const R *__restrict__ T,
                                                    bool limiters, const WorkT<R> &w, int i, int j)
{
    const int P = g.pitch;
    const int c = Ix{P}(i, j);
    if (i > g.nx || j > g.ny) return;
    const R dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const R ct1f2 = R(2) * k.CT1f;     // (unused in FP64, which reads face_ct2's table)
    if (j < g.ny) {
        const R vel = u[c], rl = rho[c - 1], rr = rho[c];
        R val = upwind(rl, rr, vel);
        if (TVD && (g.flag[c] & F_TCX))
            val += psi_surface(rho[c - 2], rl, rr, rho[c + 1], at(g.x.dc, i - 1), at(g.x.dc, i), at(g.x.dc, i + 1),
                               at(g.x.whi2, i), at(g.x.wlo2, i), vel) * (rr - rl);
        const R rdy = val * dyj;
        w.ru_dy[c] = rdy;
        w.Fx[c] = rdy * vel;
        w.DTx[c] = conductance(gam[c - 1], gam[c], at(g.x.d, i - 1), dxi, face_ct2(g.y, j, ct1f2, dyj));
    }
    if (i < g.nx) {
        const R vel = v[c], rb = rho[c - P], rt = rho[c];
        R val = upwind(rb, rt, vel);
        if (TVD && (g.flag[c] & F_TCY))
            val += psi_surface(rho[c - 2 * P], rb, rt, rho[c + P], at(g.y.dc, j - 1), at(g.y.dc, j),
                               at(g.y.dc, j + 1), at(g.y.whi2, j), at(g.y.wlo2, j), vel) * (rt - rb);
        const R rdx = val * dxi;
        w.rv_dx[c] = rdx;
        w.Fy[c] = rdx * vel;
        w.DTy[c] = conductance(gam[c - P], gam[c], at(g.y.d, j - 1), dyj, face_ct2(g.x, i, ct1f2, dxi));
    }
    const R bgc = k.B * gamma_corner(g, gam, c, i, j);
    w.Bgc[c] = bgc;
    if constexpr (std::is_same<R, double>::value) {
        // the corner's conductances of the u and v control volumes, formed
        // once here instead of by the two faces sharing the corner in the
        // assembly (the same products in the same order, so the same bits)
        w.Bgcu[c] = bgc * at(g.x.dc, i) * at(g.y.rc, j);
        w.Bgcv[c] = bgc * at(g.y.dc, j) * at(g.x.rc, i);
    }
    if (i < g.nx && j < g.ny) {
        const R bg = k.B * gam[c];
        w.Bgx[c] = bg * dyj * at(g.x.rd, i);
        w.Bgy[c] = bg * dxi * at(g.y.rd, j);
        // mass fluxes through the cell centre, the face between the u (v)
        // control volumes of faces i and i+1 (j and j+1), with the mean
        // velocity of the two faces
        const R su = u[c] + u[c + 1], sv = v[c] + v[c + P];
        w.Fbu[c] = su * half_size(g.y, j, dyj) * rho[c];
        w.Fbv[c] = sv * half_size(g.x, i, dxi) * rho[c];
        if constexpr (!std::is_same<R, float>::value) {
            w.Su[c] = su;                       // the energy source's pair sums (FP64, DF64)
            w.Sv[c] = sv;
        }
    }
    if constexpr (TVD) {
        if (limiters) face_limiters(g, u, v, T, w, c, i, j);
    }
}

// ------------------------------------------------------- explicit terms

// Face value of Eqs. pl15_11, pl31_1: the upwind node value plus psi times
// the difference across the face.  The upwind scheme (psi = 0) skips the
// correction, which IEEE arithmetic cannot drop by itself.
template <typename R, bool TVD>
__device__ __forceinline__ R face_value(R a, R b, R vel, R psi)
{
    if constexpr (TVD)
        return upwind(a, b, vel) + (b - a) * psi;
    else
        return upwind(a, b, vel);
}

// T^explicit of cell (i,j), Eq. pl31_1, all inputs at level n-1.
template <typename R, bool TVD>
__device__ R explicit_T(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &L, const WorkT<R> &w, int c, int i,
                       int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const R *T = L.T;
    const R Tp = T[c];
    const R Tw = seen_s(T, fl, c, c - 1, F_WALL, k.tau, dxi, L.rho, c, c);
    const R Te = seen_s(T, fl, c, c + 1, F_WALL, k.tau, dxi, L.rho, c, c);
    const R Ts = seen_s(T, fl, c, c - P, F_WALL, k.tau, dyj, L.rho, c, c);
    const R Tn = seen_s(T, fl, c, c + P, F_WALL, k.tau, dyj, L.rho, c, c);
    const R uw = L.u[c], ue = L.u[c + 1], vs = L.v[c], vn = L.v[c + P];
    const R Fw = w.Fx[c], Fe = w.Fx[c + 1], Fs = w.Fy[c], Fn = w.Fy[c + P];
    R pw = 0.0, pe = 0.0, ps = 0.0, pn = 0.0;
    if (TVD) {                                     // limiters of level n-1, one per face
        pe = w.psTx[c + 1];
        pw = w.psTx[c];
        pn = w.psTy[c + P];
        ps = w.psTy[c];
    }
    return -Fe * face_value<R, TVD>(Tp, Te, ue, pe) + Fw * face_value<R, TVD>(Tw, Tp, uw, pw)
           - Fn * face_value<R, TVD>(Tp, Tn, vn, pn) + Fs * face_value<R, TVD>(Ts, Tp, vs, ps);
}

// v^explicit of v face (i,j), Eq. pl15_11, level n-1.
template <typename R, bool TVD>
__device__ R explicit_v(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &L, const WorkT<R> &w, int b, int i,
                       int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *v = L.v, *u = L.u;
    const R dxi = at(g.x.d, i), dys = at(g.y.d, j - 1), dyp = at(g.y.d, j);
    const R vP = v[b];
    const R vW = seen_s(v, fl, b, b - 1, F_VWALL, k.zeta, dxi, L.rho, b - P, b);
    const R vE = seen_s(v, fl, b, b + 1, F_VWALL, k.zeta, dxi, L.rho, b - P, b);
    const R vS = v[b - P], vN = v[b + P];
    const R uw1 = u[b - P], uw2 = u[b], ue1 = u[b + 1 - P], ue2 = u[b + 1];
    const R Fw1 = w.Fx[b - P], Fw2 = w.Fx[b], Fe1 = w.Fx[b + 1 - P], Fe2 = w.Fx[b + 1];
    const R Fbs = w.Fbv[b - P], Fbn = w.Fbv[b];     // mass fluxes through the centres of cells j-1, j
    R pw1 = 0, pw2 = 0, pe1 = 0, pe2 = 0, ps = 0, pn = 0;
    if (TVD) {                                     // limiters of level n-1, one per face
        pe1 = positive(ue1) ? w.psVxU[b + 1] : w.psVxD[b + 1];
        pe2 = positive(ue2) ? w.psVxU[b + 1] : w.psVxD[b + 1];
        pw1 = positive(uw1) ? w.psVxU[b] : w.psVxD[b];
        pw2 = positive(uw2) ? w.psVxU[b] : w.psVxD[b];
        pn = w.psVy[b + P];
        ps = w.psVy[b];
    }
    return R(-0.5) * (Fe1 * face_value<R, TVD>(vP, vE, ue1, pe1) + Fe2 * face_value<R, TVD>(vP, vE, ue2, pe2))
           + R(0.5) * (Fw1 * face_value<R, TVD>(vW, vP, uw1, pw1) + Fw2 * face_value<R, TVD>(vW, vP, uw2, pw2))
           - Fbn * face_value<R, TVD>(vP, vN, Fbn, pn)
           + Fbs * face_value<R, TVD>(vS, vP, Fbs, ps);
}

// u^explicit of u face (i,j): the mirror image of Eq. pl15_11, level n-1.
template <typename R, bool TVD>
__device__ R explicit_u(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &L, const WorkT<R> &w, int a, int i,
                       int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *u = L.u, *v = L.v;
    const R dyj = at(g.y.d, j), dxw = at(g.x.d, i - 1), dxp = at(g.x.d, i);
    const R uP = u[a];
    const R uS = seen_s(u, fl, a, a - P, F_UWALL, k.zeta, dyj, L.rho, a - 1, a);
    const R uN = seen_s(u, fl, a, a + P, F_UWALL, k.zeta, dyj, L.rho, a - 1, a);
    const R uW = u[a - 1], uE = u[a + 1];
    const R vs1 = v[a - 1], vs2 = v[a], vn1 = v[a - 1 + P], vn2 = v[a + P];
    const R Fs1 = w.Fy[a - 1], Fs2 = w.Fy[a], Fn1 = w.Fy[a - 1 + P], Fn2 = w.Fy[a + P];
    const R Fbw = w.Fbu[a - 1], Fbe = w.Fbu[a];     // mass fluxes through the centres of cells i-1, i
    R pn1 = 0, pn2 = 0, ps1 = 0, ps2 = 0, pe = 0, pw = 0;
    if (TVD) {                                     // limiters of level n-1, one per face
        pn1 = positive(vn1) ? w.psUyU[a + P] : w.psUyD[a + P];
        pn2 = positive(vn2) ? w.psUyU[a + P] : w.psUyD[a + P];
        ps1 = positive(vs1) ? w.psUyU[a] : w.psUyD[a];
        ps2 = positive(vs2) ? w.psUyU[a] : w.psUyD[a];
        pe = w.psUx[a + 1];
        pw = w.psUx[a];
    }
    return R(-0.5) * (Fn1 * face_value<R, TVD>(uP, uN, vn1, pn1) + Fn2 * face_value<R, TVD>(uP, uN, vn2, pn2))
           + R(0.5) * (Fs1 * face_value<R, TVD>(uS, uP, vs1, ps1) + Fs2 * face_value<R, TVD>(uS, uP, vs2, ps2))
           - Fbe * face_value<R, TVD>(uP, uE, Fbe, pe)
           + Fbw * face_value<R, TVD>(uW, uP, Fbw, pw);
}

template <typename R, bool TVD>
__device__ __forceinline__ void explicit_terms_body(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev,
                                                    const WorkT<R> &w, int i, int j)
{
    const int c = Ix{g.pitch}(i, j);
    if (i > g.nx || j > g.ny) return;
    const uint16_t f = g.flag[c];
    if (i < g.nx && j < g.ny)
        w.Texp[c] = (f & F_FLUID) ? explicit_T<R, TVD>(g, k, prev, w, c, i, j) : R(0);
    if (j < g.ny)
        w.uexp[c] = (f & F_UACT) ? explicit_u<R, TVD>(g, k, prev, w, c, i, j) : R(0);
    if (i < g.nx)
        w.vexp[c] = (f & F_VACT) ? explicit_v<R, TVD>(g, k, prev, w, c, i, j) : R(0);
}

// ------------------------------------------------------------ temperature

// Energy source S^T_c of cell (i,j), Eq. pl29 with S^T_p = 0 (Eq. pl28):
// viscous dissipation (Eq. pl7) and pressure work; velocities off their
// nodes are bilinear interpolations, reflected across walls.
template <typename R, bool WALLS>
__device__ R energy_source(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &L, const WorkT<R> &w, int c,
                           int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *u = L.u, *v = L.v;
    const R dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const R rdx = at(g.x.rd, i), rdy = at(g.y.rd, j);
    const R dudx = (u[c + 1] - u[c]) * rdx;
    const R dvdy = (v[c + P] - v[c]) * rdy;
    // dv/dx and du/dy of the cell from the bilinear corner values: v at
    // (x^f_i, y^v_j) and (x^f_{i+1}, y^v_j), u at (x^v_i, y^f_j) and
    // (x^v_i, y^f_{j+1}), each the mean of the two face interpolations, with
    // the values across walls reflected.  With the interpolation weights
    // summing to one per face, (v_e - v_w) / dx reduces to three weighted pair
    // sums whose weights the axis tables hold (qlo, qmid, qhi).
    R dvdx, dudy;
    if constexpr (!WALLS && !std::is_same<R, float>::value) {
        // no wall in reach: the pair sums of the neighbouring cells are their
        // own v_j + v_{j+1} and u_i + u_{i+1}, which the face kernel stored
        // (the same operands in the same order, so the same bits)
        dvdx = at(g.x.qmid, i) * w.Sv[c] + at(g.x.qhi, i) * w.Sv[c + 1] - at(g.x.qlo, i) * w.Sv[c - 1];
        dudy = at(g.y.qmid, j) * w.Su[c] + at(g.y.qhi, j) * w.Su[c + P] - at(g.y.qlo, j) * w.Su[c - P];
    } else {
        const R *rho = L.rho;
        const R vW0 = seen_s<R, WALLS>(v, fl, c, c - 1, F_VWALL, k.zeta, dxi, rho, c - P, c);
        const R vW1 = seen_s<R, WALLS>(v, fl, c + P, c + P - 1, F_VWALL, k.zeta, dxi, rho, c, c + P);
        const R vE0 = seen_s<R, WALLS>(v, fl, c, c + 1, F_VWALL, k.zeta, dxi, rho, c - P, c);
        const R vE1 = seen_s<R, WALLS>(v, fl, c + P, c + P + 1, F_VWALL, k.zeta, dxi, rho, c, c + P);
        const R uS0 = seen_s<R, WALLS>(u, fl, c, c - P, F_UWALL, k.zeta, dyj, rho, c - 1, c);
        const R uS1 = seen_s<R, WALLS>(u, fl, c + 1, c + 1 - P, F_UWALL, k.zeta, dyj, rho, c, c + 1);
        const R uN0 = seen_s<R, WALLS>(u, fl, c, c + P, F_UWALL, k.zeta, dyj, rho, c - 1, c);
        const R uN1 = seen_s<R, WALLS>(u, fl, c + 1, c + 1 + P, F_UWALL, k.zeta, dyj, rho, c, c + 1);
        dvdx = at(g.x.qmid, i) * (v[c] + v[c + P]) + at(g.x.qhi, i) * (vE0 + vE1) - at(g.x.qlo, i) * (vW0 + vW1);
        dudy = at(g.y.qmid, j) * (u[c] + u[c + 1]) + at(g.y.qhi, j) * (uN0 + uN1) - at(g.y.qlo, j) * (uS0 + uS1);
    }
    const R div = dudx + dvdy, shear = dvdx + dudy;
    // 2 (dudx^2 + dvdy^2) - 2/3 div^2 = 4/3 (dudx^2 - dudx dvdy + dvdy^2)
    const R phi = R(4.0 / 3.0) * (dudx * (dudx - dvdy) + dvdy * dvdy) + shear * shear;
    const R vol = dxi * dyj;
    return (k.CT2f * L.gam[c] * phi + k.CT3f * L.p[c] * div) * vol;
}

// New temperature of fluid cell (i,j): Eq. pl30 with the implicit
// coefficients of Eq. pl31 or the explicit ones of Eq. pl31_1, conductances
// Eq. pl32 with the harmonic mean Eq. pl33.
template <typename R, bool IMPL, bool TVD, bool WALLS>
__device__ R temperature(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev, const LevelT<R> &old,
                         const WorkT<R> &w, int c, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *T = old.T;
    const R dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const R dxw = at(g.x.d, i - 1), dxe = at(g.x.d, i + 1), dys = at(g.y.d, j - 1), dyn = at(g.y.d, j + 1);
    const R Tp = T[c];
    const R Tw = seen_s<R, WALLS>(T, fl, c, c - 1, F_WALL, k.tau, dxi, old.rho, c, c);
    const R Te = seen_s<R, WALLS>(T, fl, c, c + 1, F_WALL, k.tau, dxi, old.rho, c, c);
    const R Ts = seen_s<R, WALLS>(T, fl, c, c - P, F_WALL, k.tau, dyj, old.rho, c, c);
    const R Tn = seen_s<R, WALLS>(T, fl, c, c + P, F_WALL, k.tau, dyj, old.rho, c, c);
    const R uw = old.u[c], ue = old.u[c + 1], vs = old.v[c], vn = old.v[c + P];
    const R Fw = w.Fx[c], Fe = w.Fx[c + 1], Fs = w.Fy[c], Fn = w.Fy[c + P];
    const R Dw = w.DTx[c], De = w.DTx[c + 1], Ds = w.DTy[c], Dn = w.DTy[c + P];
    // the equation divided by dt: the transient coefficients take the cell's
    // volume per unit time, the fluxes and conductances stay as they are
    const R vdt = vol_per_dt(g, k, j, dxi, dyj);
    R a1, a2, a3, a4, a0, texp;
    if (IMPL) {
        R pw = 0.0, pe = 0.0, ps = 0.0, pn = 0.0;
        if (TVD) {                                 // limiters of the level, one per face
            pw = w.psTx[c];
            pe = w.psTx[c + 1];
            ps = w.psTy[c];
            pn = w.psTy[c + P];
        }
        if constexpr (TVD) {
            a1 = pos(Fw) - Fw * pw + Dw;
            a2 = neg_part(Fe) - Fe * pe + De;
            a3 = pos(Fs) - Fs * ps + Ds;
            a4 = neg_part(Fn) - Fn * pn + Dn;
        } else {                                   // upwind: psi = 0
            a1 = pos(Fw) + Dw;
            a2 = neg_part(Fe) + De;
            a3 = pos(Fs) + Ds;
            a4 = neg_part(Fn) + Dn;
        }
        a0 = (a1 + a2 + a3 + a4 + Fe - Fw + Fn - Fs) + old.rho[c] * vdt;
        texp = R(0);
    } else {
        a1 = Dw; a2 = De; a3 = Ds; a4 = Dn;
        a0 = (a1 + a2 + a3 + a4) + old.rho[c] * vdt;
        texp = w.Texp[c];
    }
    const R sc = energy_source<R, WALLS>(g, k, old, w, c, i, j);
    R src = a1 * Tw + a2 * Te + a3 * Ts + a4 * Tn + sc;
    if constexpr (!IMPL) src += texp;
    const R rhs = src + prev.rho[c] * prev.T[c] * vdt;
    return rhs * recip(a0);
}

// ------------------------------------------------------ pseudo velocities

// u^ and d^u of u face (i,j) between fluid cells: the mirror image of
// Eqs. pl14-pl16 and pl20 (the 4/3 normal-stress factor on the x direction).
template <typename R, bool IMPL, bool TVD, bool WALLS>
__device__ void pseudo_u(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev, const LevelT<R> &old,
                         const WorkT<R> &w, int a, int i, int j, R &uhat, R &du)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *u = old.u, *v = old.v, *gam = old.gam, *rho = old.rho;
    const R dxw = at(g.x.d, i - 1), dxp = at(g.x.d, i), dyj = at(g.y.d, j);
    const R uP = u[a];
    const R uW = seen<R, WALLS>(u, fl, a, a - 1, F_UWALL), uE = seen<R, WALLS>(u, fl, a, a + 1, F_UWALL);
    const R uS = seen_s<R, WALLS>(u, fl, a, a - P, F_UWALL, k.zeta, dyj, rho, a - 1, a);
    const R uN = seen_s<R, WALLS>(u, fl, a, a + P, F_UWALL, k.zeta, dyj, rho, a - 1, a);
    const R Fbw = w.Fbu[a - 1], Fbe = w.Fbu[a];     // mass fluxes through the centres of cells i-1, i
    const R vs1 = v[a - 1], vs2 = v[a], vn1 = v[a - 1 + P], vn2 = v[a + P];
    const R Fs1 = w.Fy[a - 1], Fs2 = w.Fy[a], Fn1 = w.Fy[a - 1 + P], Fn2 = w.Fy[a + P];
    const R gcs = w.Bgc[a], gcn = w.Bgc[a + P];      // B Gamma at the corners (i, j), (i, j+1)
    const R Dxw = w.Bgx[a - 1], Dxe = w.Bgx[a];
    R Dys, Dyn;                                      // conductances of the CV's y faces (corners j, j+1)
    if constexpr (std::is_same<R, double>::value) {
        Dys = w.Bgcu[a];
        Dyn = w.Bgcu[a + P];
    } else {
        const R cx = at(g.x.dc, i);                  // centre distance of cells i-1, i: half the CV width
        Dys = gcs * cx * at(g.y.rc, j);
        Dyn = gcn * cx * at(g.y.rc, j + 1);
    }
    // dy / (2 dt): tabulated in FP64 (a load instead of an FP64 multiply)
    R vdt;
    if constexpr (std::is_same<R, double>::value)
        vdt = at(g.y.ddt, j);
    else
        vdt = dyj * k.hrdt;
    const R mass = rho[a] * dxp + rho[a - 1] * dxw;  // twice the CV mass over dy
    const R trans = mass * vdt;
    const R B23 = k.B23;
    R b = (prev.rho[a] * dxp + prev.rho[a - 1] * dxw) * vdt * prev.u[a]
               + (gcn * (vn2 - vn1) - gcs * (vs2 - vs1))
               + B23 * (gam[a - 1] * (vn1 - vs1) - gam[a] * (vn2 - vs2));
    if (nonzero(k.gx))                           // body force (uniform branch: zero in most flows)
        b += k.gx * mass * dyj * R(0.5);
    R a1, a2, a3, a4, a0, uexp;
    if (IMPL) {
        R pw = 0, pe = 0, ps1 = 0, ps2 = 0, pn1 = 0, pn2 = 0;
        if (TVD) {                                 // limiters of the level, one per face
            pw = w.psUx[a];
            pe = w.psUx[a + 1];
            ps1 = positive(vs1) ? w.psUyU[a] : w.psUyD[a];
            ps2 = positive(vs2) ? w.psUyU[a] : w.psUyD[a];
            pn1 = positive(vn1) ? w.psUyU[a + P] : w.psUyD[a + P];
            pn2 = positive(vn2) ? w.psUyU[a + P] : w.psUyD[a + P];
        }
        if constexpr (TVD) {
            a1 = pos(Fbw) - Fbw * pw + R(4.0 / 3.0) * Dxw;
            a2 = neg_part(Fbe) - Fbe * pe + R(4.0 / 3.0) * Dxe;
            a3 = R(0.5) * (pos(Fs1) - Fs1 * ps1 + pos(Fs2) - Fs2 * ps2) + Dys;
            a4 = R(0.5) * (neg_part(Fn1) - Fn1 * pn1 + neg_part(Fn2) - Fn2 * pn2) + Dyn;
        } else {                                   // upwind: psi = 0
            a1 = pos(Fbw) + R(4.0 / 3.0) * Dxw;
            a2 = neg_part(Fbe) + R(4.0 / 3.0) * Dxe;
            a3 = R(0.5) * (pos(Fs1) + pos(Fs2)) + Dys;
            a4 = R(0.5) * (neg_part(Fn1) + neg_part(Fn2)) + Dyn;
        }
        a0 = a1 + a2 + a3 + a4 + R(0.5) * (Fn2 - Fs2 + Fn1 - Fs1) + Fbe - Fbw + trans;
        uexp = R(0);
    } else {
        a1 = R(4.0 / 3.0) * Dxw; a2 = R(4.0 / 3.0) * Dxe; a3 = Dys; a4 = Dyn;
        a0 = a1 + a2 + a3 + a4 + trans;
        uexp = w.uexp[a];
    }
    const R r = recip(a0);
    R src = a1 * uW + a2 * uE + a3 * uS + a4 * uN + b;
    if constexpr (!IMPL) src += uexp;
    uhat = src * r;
    // A = 1/2 for every gas model of this solver (Eq. pl37, and the ideal-gas
    // mapping of the coefficients): in FP64 A dy is the tabulated half height
    // (the same value, no multiply)
    R Ady;
    if constexpr (std::is_same<R, double>::value)
        Ady = half_size(g.y, j, dyj);
    else
        Ady = k.A * dyj;
    du = Ady * r;
}

// v^ and d^v of v face (i,j) between fluid cells, Eqs. pl14-pl16, pl21
// (implicit, Eq. pl15; explicit, Eq. pl15_11).
template <typename R, bool IMPL, bool TVD, bool WALLS>
__device__ void pseudo_v(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev, const LevelT<R> &old,
                         const WorkT<R> &w, int b, int i, int j, R &vhat, R &dv)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const R *u = old.u, *v = old.v, *gam = old.gam, *rho = old.rho;
    const R dys = at(g.y.d, j - 1), dyp = at(g.y.d, j), dxi = at(g.x.d, i);
    const R vP = v[b];
    const R vW = seen_s<R, WALLS>(v, fl, b, b - 1, F_VWALL, k.zeta, dxi, rho, b - P, b);
    const R vE = seen_s<R, WALLS>(v, fl, b, b + 1, F_VWALL, k.zeta, dxi, rho, b - P, b);
    const R vS = seen<R, WALLS>(v, fl, b, b - P, F_VWALL), vN = seen<R, WALLS>(v, fl, b, b + P, F_VWALL);
    const R Fbs = w.Fbv[b - P], Fbn = w.Fbv[b];     // mass fluxes through the centres of cells j-1, j
    const R uw1 = u[b - P], uw2 = u[b], ue1 = u[b + 1 - P], ue2 = u[b + 1];
    const R Fw1 = w.Fx[b - P], Fw2 = w.Fx[b], Fe1 = w.Fx[b + 1 - P], Fe2 = w.Fx[b + 1];
    const R gcw = w.Bgc[b], gce = w.Bgc[b + 1];      // B Gamma at the corners (i, j), (i+1, j)
    R Dxw, Dxe;                                      // conductances of the CV's x faces (corners i, i+1)
    if constexpr (std::is_same<R, double>::value) {
        Dxw = w.Bgcv[b];
        Dxe = w.Bgcv[b + 1];
    } else {
        const R cy = at(g.y.dc, j);                  // centre distance of cells j-1, j: half the CV height
        Dxw = gcw * cy * at(g.x.rc, i);
        Dxe = gce * cy * at(g.x.rc, i + 1);
    }
    const R Dys = w.Bgy[b - P], Dyn = w.Bgy[b];
    R vdt;
    if constexpr (std::is_same<R, double>::value)
        vdt = at(g.x.ddt, i);
    else
        vdt = dxi * k.hrdt;
    const R mass = rho[b] * dyp + rho[b - P] * dys;  // twice the CV mass over dx
    const R trans = mass * vdt;
    const R B23 = k.B23;
    R bsrc = (prev.rho[b] * dyp + prev.rho[b - P] * dys) * vdt * prev.v[b]
                  + (gce * (ue2 - ue1) - gcw * (uw2 - uw1))
                  + B23 * (gam[b - P] * (ue1 - uw1) - gam[b] * (ue2 - uw2));
    if (nonzero(k.gy))                           // body force (uniform branch: zero in most flows)
        bsrc += k.gy * mass * dxi * R(0.5);
    R a1, a2, a3, a4, a0, vexp;
    if (IMPL) {
        R pw1 = 0, pw2 = 0, pe1 = 0, pe2 = 0, ps = 0, pn = 0;
        if (TVD) {                                 // limiters of the level, one per face
            pw1 = positive(uw1) ? w.psVxU[b] : w.psVxD[b];
            pw2 = positive(uw2) ? w.psVxU[b] : w.psVxD[b];
            pe1 = positive(ue1) ? w.psVxU[b + 1] : w.psVxD[b + 1];
            pe2 = positive(ue2) ? w.psVxU[b + 1] : w.psVxD[b + 1];
            ps = w.psVy[b];
            pn = w.psVy[b + P];
        }
        if constexpr (TVD) {
            a1 = R(0.5) * (pos(Fw2) - Fw2 * pw2 + pos(Fw1) - Fw1 * pw1) + Dxw;
            a2 = R(0.5) * (neg_part(Fe2) - Fe2 * pe2 + neg_part(Fe1) - Fe1 * pe1) + Dxe;
            a3 = pos(Fbs) - Fbs * ps + R(4.0 / 3.0) * Dys;
            a4 = neg_part(Fbn) - Fbn * pn + R(4.0 / 3.0) * Dyn;
        } else {                                   // upwind: psi = 0
            a1 = R(0.5) * (pos(Fw2) + pos(Fw1)) + Dxw;
            a2 = R(0.5) * (neg_part(Fe2) + neg_part(Fe1)) + Dxe;
            a3 = pos(Fbs) + R(4.0 / 3.0) * Dys;
            a4 = neg_part(Fbn) + R(4.0 / 3.0) * Dyn;
        }
        a0 = a1 + a2 + a3 + a4 + R(0.5) * (Fe2 - Fw2 + Fe1 - Fw1) + Fbn - Fbs + trans;
        vexp = R(0);
    } else {
        a1 = Dxw; a2 = Dxe; a3 = R(4.0 / 3.0) * Dys; a4 = R(4.0 / 3.0) * Dyn;
        a0 = a1 + a2 + a3 + a4 + trans;
        vexp = w.vexp[b];
    }
    const R r = recip(a0);
    R src = a1 * vW + a2 * vE + a3 * vS + a4 * vN + bsrc;
    if constexpr (!IMPL) src += vexp;
    vhat = src * r;
    R Adx;
    if constexpr (std::is_same<R, double>::value)
        Adx = half_size(g.x, i, dxi);
    else
        Adx = k.A * dxi;
    dv = Adx * r;
}

// The pressure equation's face terms of Eq. pl24, formed once per face where
// the pseudo velocity and d are made (FP64; the pressure kernel would form
// each twice, once for each cell sharing the face): the coefficient
// a^p = rho^f area d replaces rho^f area in `ra`, the source flux
// b^p = rho^f area u^ goes to `bp`.  The same products as the pressure kernel
// formed, so the same bits.
__device__ __forceinline__ void pressure_face_terms(double *ra, double *bp, int c, double uh, double d)
{
    const double r = ra[c];
    ra[c] = r * d;
    bp[c] = r * uh;
}

template <typename R, bool IMPL, bool TVD, bool WALLS>
__device__ __forceinline__ void assemble_at(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev,
                                            const LevelT<R> &old, R *__restrict__ T_out, const WorkT<R> &w, int c,
                                            uint16_t f, int i, int j)
{
    if (i < g.nx && j < g.ny && (f & F_FLUID)) {
        const R Tn = temperature<R, IMPL, TVD, WALLS>(g, k, prev, old, w, c, i, j);
        T_out[c] = Tn;
    }
    if (j < g.ny) {
        R uh = old.u[c], d = R(0);            // faces that are not unknowns: stored u, d = 0
        if (f & F_UACT)
            pseudo_u<R, IMPL, TVD, WALLS>(g, k, prev, old, w, c, i, j, uh, d);
        w.uhat[c] = uh;
        w.du[c] = d;
        if constexpr (std::is_same<R, double>::value)
            pressure_face_terms(w.ru_dy, w.bpx, c, uh, d);
    }
    if (i < g.nx) {
        R vh = old.v[c], d = R(0);
        if (f & F_VACT)
            pseudo_v<R, IMPL, TVD, WALLS>(g, k, prev, old, w, c, i, j, vh, d);
        w.vhat[c] = vh;
        w.dv[c] = d;
        if constexpr (std::is_same<R, double>::value)
            pressure_face_terms(w.rv_dx, w.bpy, c, vh, d);
    }
}

// One thread per position: T of the cell, u^/d^u of the u face, v^/d^v of
// the v face.  The new T goes to T_out, in the compute precision (the mixed
// path's FP64 view of it is filled when the state is read: widen_mixed_at).
template <typename R, bool IMPL, bool TVD>
__device__ __forceinline__ void assemble_body(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev,
                                              const LevelT<R> &old, R *__restrict__ T_out, const WorkT<R> &w,
                                              int i, int j)
{
    if (i > g.nx || j > g.ny) return;
    const int c = Ix{g.pitch}(i, j);
    const uint16_t f = g.flag[c];
    // Positions of wall-free 32-wide row segments take the variant without
    // wall reflections (fewer instructions).  The choice depends on the
    // position only, never on how threads form warps, so every tiling gives
    // the same bits; with 32-wide tiles it is uniform across each warp.
    if (std::is_same<R, double>::value && (f & F_INTERIOR)) {
        // Every cell within two of the segment is fluid, so the position is a
        // fluid cell inside the domain with both of its faces unknowns: all
        // three equations apply.  In FP64 they are evaluated first and stored
        // after, so that no store separates the loads of one equation from
        // those of the next (the compiler cannot move a load above a store it
        // cannot prove apart) and their memory latencies overlap: 1.579 ->
        // 1.511 ms per launch on the 4864x1216 channel.  The FP32 and
        // double-float assemblies, held to 64 registers, would spill for it
        // (measured: mixed -4 %, double-float -12 %) and keep the branches.
        const R Tn = temperature<R, IMPL, TVD, false>(g, k, prev, old, w, c, i, j);
        R uh, du, vh, dv;
        pseudo_u<R, IMPL, TVD, false>(g, k, prev, old, w, c, i, j, uh, du);
        pseudo_v<R, IMPL, TVD, false>(g, k, prev, old, w, c, i, j, vh, dv);
        T_out[c] = Tn;
        w.uhat[c] = uh;
        w.du[c] = du;
        w.vhat[c] = vh;
        w.dv[c] = dv;
        if constexpr (std::is_same<R, double>::value) {
            pressure_face_terms(w.ru_dy, w.bpx, c, uh, du);
            pressure_face_terms(w.rv_dx, w.bpy, c, vh, dv);
        }
    } else if (f & F_INTERIOR) {
        assemble_at<R, IMPL, TVD, false>(g, k, prev, old, T_out, w, c, f, i, j);
    } else {
        assemble_at<R, IMPL, TVD, true>(g, k, prev, old, T_out, w, c, f, i, j);
    }
}

// ---------------------------------------------------------------- pressure

// Eqs. pl23, pl24 with the new T (point Jacobi in p^old), then rho = p/T
// (Eq. pl5) and Gamma = T^omega, with the p and T residual maxima.  The
// divisions by T and a^p_0 use the sweep's reciprocal.
template <typename R>
__device__ __forceinline__ void pressure_body(const GeoT<R> &g, const CoefT<R> &k, const LevelT<R> &prev,
                                              const LevelT<R> &old, const LevelT<R> &nw, const WorkT<R> &w,
                                              unsigned long long *res, int i, int j, bool own)
{
    const int P = g.pitch;
    unsigned long long rp = 0, rT = 0;
    if (i < g.nx && j < g.ny) {
        const int c = Ix{P}(i, j);
        if (g.flag[c] & F_FLUID) {
            const R dxi = at(g.x.d, i), dyj = at(g.y.d, j);
            // coefficients a^p and source fluxes b^p of the four faces: stored
            // by the FP64 assembly; formed here from rho^u dy and rho^v dx (face
            // kernel) and u^, d by the double-float sweep
            R apw, ape, aps, apn, bpw, bpe, bps, bpn;
            if constexpr (std::is_same<R, double>::value) {
                apw = w.ru_dy[c];
                ape = w.ru_dy[c + 1];
                aps = w.rv_dx[c];
                apn = w.rv_dx[c + P];
                bpw = w.bpx[c];
                bpe = w.bpx[c + 1];
                bps = w.bpy[c];
                bpn = w.bpy[c + P];
            } else {
                const R ru_w = w.ru_dy[c], ru_e = w.ru_dy[c + 1], rv_s = w.rv_dx[c], rv_n = w.rv_dx[c + P];
                apw = ru_w * w.du[c];
                ape = ru_e * w.du[c + 1];
                aps = rv_s * w.dv[c];
                apn = rv_n * w.dv[c + P];
                bpw = ru_w * w.uhat[c];
                bpe = ru_e * w.uhat[c + 1];
                bps = rv_s * w.vhat[c];
                bpn = rv_n * w.vhat[c + P];
            }
            const R Tn = nw.T[c], inv_T = recip(Tn);
            // Eqs. pl23, pl24 divided by dt (the transient terms take the
            // cell's volume per unit time): the neighbour sum accumulates
            // onto the source
            const R vdt = vol_per_dt(g, k, j, dxi, dyj);
            const R ap0 = vdt * inv_T + (apw + ape + aps + apn);
            const R bp = prev.rho[c] * vdt - (bpe - bpw + bpn - bps);
            const R pn = ((((bp + apw * old.p[c - 1]) + ape * old.p[c + 1]) + aps * old.p[c - P]) + apn * old.p[c + P])
                         * recip(ap0);
            nw.p[c] = pn;
            nw.rho[c] = pn * inv_T;
            nw.gam[c] = gamma_of(Tn, k.omega);
            rp = res_key(pn - old.p[c]);
            rT = res_key(Tn - old.T[c]);
        }
    }
    if (!own) rp = rT = 0;
    block_max2(rp, rT, &res[2], &res[3]);
}

// -------------------------------------------------------------- velocity

// Outflow side (zero gradient): the thread of column nx-1 copies its new
// values into the ghost columns nx, nx+1 (cells, v) and nx, nx+1, nx+2 (u).
template <typename R>
__device__ __forceinline__ void outflow_copy(int j, int ny, int c, LevelT<R> L)
{
    if (j < ny) {
        R *sc[4] = {L.p, L.T, L.rho, L.gam};
        for (int q = 0; q < 4; q++) {
            const R x = sc[q][c];
            sc[q][c + 1] = x;
            sc[q][c + 2] = x;
        }
        const R un = L.u[c];
        L.u[c + 1] = un;
        L.u[c + 2] = un;
        L.u[c + 3] = un;
    }
    const R vn = L.v[c];
    L.v[c + 1] = vn;
    L.v[c + 2] = vn;
}

// The outflow copies of p and rho alone: the FP64 values the mixed path's
// sweep reads (its FP64 u, v, T and Gamma are filled when the state is read).
__device__ __forceinline__ void outflow_copy_p_rho(int j, int ny, int c, const Level &L)
{
    if (j < ny) {
        const double p = L.p[c], rho = L.rho[c];
        L.p[c + 1] = p;
        L.p[c + 2] = p;
        L.rho[c + 1] = rho;
        L.rho[c + 2] = rho;
    }
}

// Eqs. pl18, pl19: velocities of the face unknowns from the new pressure,
// then the outflow ghost copies of the row.
template <typename R>
__device__ __forceinline__ void velocity_body(const GeoT<R> &g, const LevelT<R> &old, const LevelT<R> &nw,
                                              const WorkT<R> &w, unsigned long long *res, int east_outflow, int i,
                                              int j, bool own)
{
    const int P = g.pitch;
    unsigned long long ru = 0, rv = 0;
    if (i <= g.nx && j <= g.ny) {
        const int c = Ix{P}(i, j);
        const uint16_t f = g.flag[c];
        if constexpr (std::is_same<R, double>::value) {
            // FP64: every operand loaded before the flag decides what is
            // stored, so the loads do not wait for it (-5 % on this kernel;
            // the double-float sweep, slower with it, keeps the loads behind)
            const R uh = w.uhat[c], du = w.du[c], vh = w.vhat[c], dv = w.dv[c], uo = old.u[c], vo = old.v[c];
            const R pc = nw.p[c], pw = nw.p[c - 1], ps = nw.p[c - P];
            if (j < g.ny && (f & F_UACT)) {
                const R un = uh - du * (pc - pw);
                nw.u[c] = un;
                ru = res_key(un - uo);
            }
            if (i < g.nx && (f & F_VACT)) {
                const R vn = vh - dv * (pc - ps);
                nw.v[c] = vn;
                rv = res_key(vn - vo);
            }
        } else {
            if (j < g.ny && (f & F_UACT)) {
                const R un = w.uhat[c] - w.du[c] * (nw.p[c] - nw.p[c - 1]);
                nw.u[c] = un;
                ru = res_key(un - old.u[c]);
            }
            if (i < g.nx && (f & F_VACT)) {
                const R vn = w.vhat[c] - w.dv[c] * (nw.p[c] - nw.p[c - P]);
                nw.v[c] = vn;
                rv = res_key(vn - old.v[c]);
            }
        }
        if (east_outflow && i == g.nx - 1)
            outflow_copy(j, g.ny, c, nw);
    }
    if (!own) ru = rv = 0;
    block_max2(ru, rv, &res[0], &res[1]);
}

// --------------------------------------------------------- mixed precision

// Mixed precision, pressure: the coefficients of Eqs. pl23, pl24 come from
// the FP32 assembly (FP32 rho^u, d, u^ and the new T); the accumulation of
// the neighbour pressures and the source, the division by a^p_0, the
// equation of state rho = p/T and the residual of p are FP64.  The FP64
// reciprocals start from the FP32 reciprocal and take one Newton step
// (relative error below 1e-14).  Gamma = T^omega is a coefficient: FP32.
// T carries FP32 values in this path, so its residual difference is formed
// exactly in FP32.
__device__ __forceinline__ void pressure_mixed_body(const Geo &g, const Coef &k, const GeoT<float> &g32,
                                                    const CoefT<float> &k32, const Level &prev, const Level &old,
                                                    const Level &nw, const LevelT<float> &old32,
                                                    const LevelT<float> &nw32, const WorkT<float> &w,
                                                    unsigned long long *res, int i, int j, bool own)
{
    const int P = g.pitch;
    unsigned long long rp = 0, rT = 0;
    if (i < g.nx && j < g.ny) {
        const int c = Ix{P}(i, j);
        // evaluated for every cell, the flag deciding only what is stored, so
        // the loads do not wait for it (-3 % on this kernel)
        const bool fluid = (g.flag[c] & F_FLUID) != 0;
        {
            const float dxi = at(g32.x.d, i), dyj = at(g32.y.d, j);
            const float ru_w = w.ru_dy[c], ru_e = w.ru_dy[c + 1], rv_s = w.rv_dx[c], rv_n = w.rv_dx[c + P];
            const float apw = ru_w * w.du[c], ape = ru_e * w.du[c + 1];
            const float aps = rv_s * w.dv[c], apn = rv_n * w.dv[c + P];
            const float bpw = ru_w * w.uhat[c], bpe = ru_e * w.uhat[c + 1];
            const float bps = rv_s * w.vhat[c], bpn = rv_n * w.vhat[c + P];
            const float T32 = nw32.T[c];
            const double Tn = widen(T32);
            // divided by dt, as the FP64 pressure kernel: the cell's volume
            // per unit time in the transient terms, a coefficient assembled
            // in FP32 like the others; the source accumulates it in FP64
            // (the FP32 product widens exactly)
            const float vdt = dxi * at(g32.y.dt1, j);
            const float ap0 = vdt / T32 + (apw + ape + aps + apn);
            const float div = (bpe - bpw) + (bpn - bps);
            const double bp = fma(prev.rho[c], widen(vdt), widen(-div));
            double num = fma(widen(apw), old.p[c - 1], bp);
            num = fma(widen(ape), old.p[c + 1], num);
            num = fma(widen(aps), old.p[c - P], num);
            num = fma(widen(apn), old.p[c + P], num);
            const double a0 = widen(ap0);
            double r = widen(1.0f / ap0);
            r = fma(r, fma(-a0, r, 1.0), r);
            const double pn = num * r;
            double rt = widen(1.0f / T32);
            rt = fma(rt, fma(-Tn, rt, 1.0), rt);
            const double rho = pn * rt;
            const float gm = (k32.omega == 0.5f) ? sqrtf(T32) : powf(T32, k32.omega);
            const double po = old.p[c];
            const float To = old32.T[c];
            if (fluid) {
                nw.p[c] = pn;
                nw.rho[c] = rho;
                nw32.p[c] = narrow(pn);
                nw32.rho[c] = narrow(rho);
                nw32.gam[c] = gm;
                rp = ordered_bits(pn - po);
                rT = ordered_bits(widen(T32 - To));
            }
        }
    }
    if (!own) rp = rT = 0;
    block_max2(rp, rT, &res[2], &res[3]);
}

// Mixed precision, Eqs. pl18, pl19: FP32 correction of the FP32 pseudo
// velocities by the FP64 pressure difference.  u and v carry FP32 values in
// this path: their residual differences are formed in FP32 and reduced as
// FP64 bit patterns, and the FP64 state holds them only once it is read
// (widen_mixed_at).
__device__ __forceinline__ void velocity_mixed_body(const Geo &g, const Level &nw, const LevelT<float> &old32,
                                                    const LevelT<float> &nw32, const WorkT<float> &w,
                                                    unsigned long long *res, int east_outflow, int i, int j,
                                                    bool own)
{
    const int P = g.pitch;
    unsigned long long ru = 0, rv = 0;
    if (i <= g.nx && j <= g.ny) {
        const int c = Ix{P}(i, j);
        const uint16_t f = g.flag[c];
        // every operand is loaded before the flag decides what is stored, so
        // the loads do not wait for the flag (every index is inside the
        // padded arrays for positions up to (nx, ny)): -9 % on this kernel
        const float uh = w.uhat[c], du = w.du[c], vh = w.vhat[c], dv = w.dv[c], uo = old32.u[c], vo = old32.v[c];
        const double pc = nw.p[c], pw = nw.p[c - 1], ps = nw.p[c - P];
        if (j < g.ny && (f & F_UACT)) {
            const float un32 = uh - du * narrow(pc - pw);
            nw32.u[c] = un32;
            ru = ordered_bits(widen(un32 - uo));
        }
        if (i < g.nx && (f & F_VACT)) {
            const float vn32 = vh - dv * narrow(pc - ps);
            nw32.v[c] = vn32;
            rv = ordered_bits(widen(vn32 - vo));
        }
        if (east_outflow && i == g.nx - 1) {
            outflow_copy_p_rho(j, g.ny, c, nw);
            outflow_copy(j, g.ny, c, nw32);
        }
    }
    if (!own) ru = rv = 0;
    block_max2(ru, rv, &res[0], &res[1]);
}

// The FP64 view of a mixed-precision level at position (i, j): u, v, T and
// Gamma, which the sweep keeps in FP32 only, widened (exactly) where the
// sweep computes them -- T and Gamma of fluid cells, u and v of the face
// unknowns -- then, on an outflow side, the ghost copies of column nx - 1.
// The other positions keep their FP64 values, which the sweep never changes,
// so the view holds what a sweep storing FP64 copies would have stored.
__device__ __forceinline__ void widen_mixed_at(const Geo &g, const Level &L, const LevelT<float> &S,
                                               int east_outflow, int i, int j)
{
    if (i > g.nx || j > g.ny) return;
    const int c = Ix{g.pitch}(i, j);
    const uint16_t f = g.flag[c];
    if (i < g.nx && j < g.ny && (f & F_FLUID)) {
        L.T[c] = widen(S.T[c]);
        L.gam[c] = widen(S.gam[c]);
    }
    if (j < g.ny && (f & F_UACT)) L.u[c] = widen(S.u[c]);
    if (i < g.nx && (f & F_VACT)) L.v[c] = widen(S.v[c]);
    if (east_outflow && i == g.nx - 1) outflow_copy(j, g.ny, c, L);
}

// ------------------------------------------------------- tile-list kernels

// The equation kernels walk a tile list (BatchPlan): the tiles of one or
// more problems, each tile tx x ty threads of one problem, taken by the
// resident CTAs in turn.  A single problem is a list of one; every caller
// runs these same kernels, so a problem's arithmetic does not depend on what
// else shares the launch or on the tile shape.
// Where a kernel reads the descriptor of the tile's problem from (ONE):
// - staged in shared memory (ONE false): from the launch parameters when the
//   list holds one problem, else from the device array, once per problem a
//   CTA meets;
// - read in place from the launch parameters (ONE true, a list of one
//   problem): no copy and no barrier before the first tile.
// On the 4864 x 1216 channel the second made the FP32 (mixed) sweep 8 % and
// the double-float sweep 12 % faster and the FP64 sweep 2 % slower, so the
// host takes it for one problem in FP32 or double-float.  Both give the same
// bits.
template <bool ONE, typename F>
__device__ __forceinline__ void for_tiles(const BatchPlan &bp, F &&f)
{
    auto tile = [&](const Inst &I, int t) {
        const int lt = t - I.tile0;
        int i = I.x0 + (lt % I.tiles_x) * bp.tx + threadIdx.x;
        const int j = (lt / I.tiles_x) * bp.ty + threadIdx.y;
        if (I.x_stop > 0 && i >= I.x_stop) i = I.g.nx + 1;   // beyond every body's range
        f(I, i, j);
    };
    if constexpr (ONE) {
        for (int t = blockIdx.x; t < bp.n_tiles; t += gridDim.x) tile(bp.one, t);
    } else {
        static_assert(sizeof(Inst) % 8 == 0, "Inst is copied as 8-byte words");
        constexpr int kWords = sizeof(Inst) / 8;
        __shared__ __align__(16) Inst sI;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
        int have = -1;
        for (int t = blockIdx.x; t < bp.n_tiles; t += gridDim.x) {
            const int q = bp.n_inst == 1 ? 0 : bp.tile_inst[t];
            if (q != have) {
                if (have >= 0) __syncthreads();           // the previous problem's tile is done
                const unsigned long long *src = bp.n_inst == 1
                                                    ? reinterpret_cast<const unsigned long long *>(&bp.one)
                                                    : reinterpret_cast<const unsigned long long *>(bp.inst + q);
                unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sI);
                for (int w = tid; w < kWords; w += nthr) dst[w] = src[w];
                __syncthreads();
                have = q;
            }
            tile(sI, t);
        }
    }
}

// Whether column i counts for the residual maxima of the descriptor's problem
// (every column of a whole problem; the owned columns of an x-strip).
__device__ __forceinline__ bool owns(const Inst &I, int i)
{
    return i >= I.own0 && (I.own_stop == 0 || i < I.own_stop);
}

// The residual words of every problem of the list to 0.  The face kernel
// does this in its first CTA: it runs at the start of every loop-2 iteration
// (for the first iteration of an explicit step, as part of the explicit
// terms), before the pressure and velocity kernels accumulate the maxima, and
// after the previous iteration's velocity kernel has finished.  (A separate
// memset or kernel for it costs a node of the step graph.)
__device__ __forceinline__ void reset_residuals(const BatchPlan &bp)
{
    if (blockIdx.x != 0) return;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    for (int q = tid; q < bp.n_inst * 4; q += nthr) bp.inst[q >> 2].w.res[q & 3] = 0ull;
}

// ------------------------------------------------------------------ phases

// The phases of one loop-2 iteration over a tile list, each what one
// per-phase kernel of phase_kernels.cuh runs; the persistent step kernel
// (k_step) runs them one after another with a grid barrier between them.
template <int PREC, bool TVD, bool ONE = false>
__device__ __forceinline__ void faces_phase(const BatchPlan &bp, int level, int limiters)
{
    reset_residuals(bp);
    for_tiles<ONE>(bp, [&](const Inst &I, int i, int j) {
        if constexpr (PREC == PREC_MIXED) {
            const LevelT<float> &L = I.lv32[level];
            face_densities_body<float, TVD>(I.g32, I.k32, L.u, L.v, L.rho, L.gam, L.T, limiters, I.w32, i, j);
        } else if constexpr (PREC == PREC_DF64) {
            const LevelT<df64> &L = I.lvdf[level];
            face_densities_body<df64, TVD>(I.gdf, I.kdf, L.u, L.v, L.rho, L.gam, L.T, limiters, I.wdf, i, j);
        } else {
            const Level &L = I.lv[level];
            face_densities_body<double, TVD>(I.g, I.k, L.u, L.v, L.rho, L.gam, L.T, limiters, I.w, i, j);
        }
    });
}

template <int PREC, bool TVD, bool ONE = false>
__device__ __forceinline__ void explicit_phase(const BatchPlan &bp, int prev)
{
    for_tiles<ONE>(bp, [&](const Inst &I, int i, int j) {
        if constexpr (PREC == PREC_MIXED)
            explicit_terms_body<float, TVD>(I.g32, I.k32, I.lv32[prev], I.w32, i, j);
        else if constexpr (PREC == PREC_DF64)
            explicit_terms_body<df64, TVD>(I.gdf, I.kdf, I.lvdf[prev], I.wdf, i, j);
        else
            explicit_terms_body<double, TVD>(I.g, I.k, I.lv[prev], I.w, i, j);
    });
}

template <int PREC, bool IMPL, bool TVD, bool ONE = false>
__device__ __forceinline__ void assemble_phase(const BatchPlan &bp, int prev, int old, int nw)
{
    for_tiles<ONE>(bp, [&](const Inst &I, int i, int j) {
        if constexpr (PREC == PREC_MIXED)
            assemble_body<float, IMPL, TVD>(I.g32, I.k32, I.lv32[prev], I.lv32[old], I.lv32[nw].T, I.w32, i, j);
        else if constexpr (PREC == PREC_DF64)
            assemble_body<df64, IMPL, TVD>(I.gdf, I.kdf, I.lvdf[prev], I.lvdf[old], I.lvdf[nw].T, I.wdf, i, j);
        else
            assemble_body<double, IMPL, TVD>(I.g, I.k, I.lv[prev], I.lv[old], I.lv[nw].T, I.w, i, j);
    });
}

template <int PREC, bool ONE = false>
__device__ __forceinline__ void pressure_phase(const BatchPlan &bp, int prev, int old, int nw)
{
    for_tiles<ONE>(bp, [&](const Inst &I, int i, int j) {
        if constexpr (PREC == PREC_MIXED)
            pressure_mixed_body(I.g, I.k, I.g32, I.k32, I.lv[prev], I.lv[old], I.lv[nw], I.lv32[old], I.lv32[nw],
                                I.w32, I.w.res, i, j, owns(I, i));
        else if constexpr (PREC == PREC_DF64)
            pressure_body<df64>(I.gdf, I.kdf, I.lvdf[prev], I.lvdf[old], I.lvdf[nw], I.wdf, I.w.res, i, j,
                                owns(I, i));
        else
            pressure_body<double>(I.g, I.k, I.lv[prev], I.lv[old], I.lv[nw], I.w, I.w.res, i, j, owns(I, i));
    });
}

template <int PREC, bool ONE = false>
__device__ __forceinline__ void velocity_phase(const BatchPlan &bp, int old, int nw)
{
    for_tiles<ONE>(bp, [&](const Inst &I, int i, int j) {
        if constexpr (PREC == PREC_MIXED)
            velocity_mixed_body(I.g, I.lv[nw], I.lv32[old], I.lv32[nw], I.w32, I.w.res, I.east_outflow, i, j,
                                owns(I, i));
        else if constexpr (PREC == PREC_DF64)
            velocity_body<df64>(I.gdf, I.lvdf[old], I.lvdf[nw], I.wdf, I.w.res, I.east_outflow, i, j, owns(I, i));
        else
            velocity_body<double>(I.g, I.lv[old], I.lv[nw], I.w, I.w.res, I.east_outflow, i, j, owns(I, i));
    });
}

}  // namespace
}  // namespace stg
