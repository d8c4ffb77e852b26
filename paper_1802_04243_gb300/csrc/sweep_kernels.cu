// sweep_kernels.cu -- FP64 CUDA kernels of one SIMPLE-TS time step
// (K. S. Shterev, arXiv:1802.04243, Sections 3.1 and 3.2) for sm_103a.
//
// One loop-2 iteration (Section 3.1, Figs. 1 and 2, GPU column) runs as
//   k_face_densities   rho^u, rho^v of every face            (Eqs. pl8-pl11)
//   k_assemble         T, u^/d^u, v^/d^v of every node         (Eqs. pl14-pl16, pl20, pl21, pl28-pl33)
//   k_pressure         p, rho = p/T, Gamma = T^omega, |dp|, |dT| (Eqs. pl23, pl24, pl5)
//   k_velocity         u, v from the new p, |du|, |dv|          (Eqs. pl18, pl19)
//   k_ghost_*          outflow / symmetry ghost copies
// and, once per step for the explicit scheme, k_explicit_terms (Eqs. pl15_11,
// pl31_1 and the u mirror).  Each thread owns one grid position (i, j) and
// the cell, the u face and the v face with that index.
//
// Boundary rules: wall ghost and obstacle cells hold the wall state; a
// temperature or tangential velocity read across a wall is reflected about
// the stored wall value (2 phi_wall - phi_reader); TVD corrections apply only
// where the flag of the face says all four stencil nodes are unknowns.
#include <cuda_runtime.h>
#include <math.h>

#include "stg_common.cuh"

namespace stg {
namespace {

constexpr int BX = 32, BY = 8;

struct Ix {
    int P;
    __device__ __forceinline__ int operator()(int i, int j) const { return (j + G) * P + (i + G); }
};

__device__ __forceinline__ double at(const double *a, int i) { return a[i + G]; }

// ---------------------------------------------------------------- limiter

// Van Leer psi(r) = (r + |r|)/(1 + r) for r = num/den; 0 unless num and den
// share a sign (a zero denominator falls back to first order).
__device__ __forceinline__ double van_leer(double num, double den)
{
    return (num * den > 0.0) ? 2.0 * num / (num + den) : 0.0;
}

// Eq. pl15_2: correction at the face between nodes 2 and 3; d1..d4 are the
// cell sizes of the four nodes.
__device__ __forceinline__ double psi_surface(double f1, double f2, double f3, double f4,
                                              double d1, double d2, double d3, double d4, double vel)
{
    if (vel > 0.0)
        return d2 / (d2 + d3) * van_leer((d2 + d3) * (f2 - f1), (d1 + d2) * (f3 - f2));
    return -d3 / (d2 + d3) * van_leer((d2 + d3) * (f4 - f3), (d3 + d4) * (f3 - f2));
}

// Eq. pl15_1: face midway between nodes 2 and 3; d1..d3 the node distances.
__device__ __forceinline__ double psi_centre(double f1, double f2, double f3, double f4,
                                             double d1, double d2, double d3, double vel)
{
    if (vel > 0.0)
        return 0.5 * van_leer(d2 * (f2 - f1), d1 * (f3 - f2));
    return -0.5 * van_leer(d2 * (f4 - f3), d3 * (f3 - f2));
}

__device__ __forceinline__ double upwind(double a, double b, double vel) { return vel > 0.0 ? a : b; }
__device__ __forceinline__ double pos(double x) { return fmax(0.0, x); }

// Value of node m seen from node a: reflected about the stored wall value when
// the flag of m carries `wall_bit`.
__device__ __forceinline__ double seen(const double *f, const uint16_t *flag, int a, int m, uint32_t wall_bit)
{
    double fm = f[m];
    return (flag[m] & wall_bit) ? 2.0 * fm - f[a] : fm;
}

// Gamma at the corner (x^f_i, y^f_j): bilinear in the four cell centres.
__device__ __forceinline__ double gamma_corner(const Geo &g, const double *gam, int c, int i, int j)
{
    const int P = g.pitch;
    double lo = at(g.x.wlo, i) * gam[c - P - 1] + at(g.x.whi, i) * gam[c - P];
    double hi = at(g.x.wlo, i) * gam[c - 1] + at(g.x.whi, i) * gam[c];
    return at(g.y.wlo, j) * lo + at(g.y.whi, j) * hi;
}

// Eq. pl33: distance-weighted harmonic mean of Gamma^lambda across a face
// between a node of size da and one of size db.
__device__ __forceinline__ double harmonic(double ga, double gb, double da, double db)
{
    return (da + db) * ga * gb / (da * gb + db * ga);
}

// ------------------------------------------------------ residual reduction

__device__ __forceinline__ unsigned long long ordered(double x)
{
    // |x| as an unsigned integer: ordered like the value, NaN above infinity
    return (unsigned long long)__double_as_longlong(fabs(x));
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
}

// ------------------------------------------------------- face densities

// rho^u at u face (i,j) and rho^v at v face (i,j), Eqs. pl10, pl11, written as
// the upwind value plus psi_s times the difference across the face.
template <bool TVD>
__global__ void __launch_bounds__(BX *BY) k_face_densities(Geo g, const double *__restrict__ u,
                                                            const double *__restrict__ v,
                                                            const double *__restrict__ rho,
                                                            double *__restrict__ rho_u,
                                                            double *__restrict__ rho_v)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int P = g.pitch;
    const int c = Ix{P}(i, j);
    if (i <= g.nx && j < g.ny) {
        const double vel = u[c], rl = rho[c - 1], rr = rho[c];
        double val = upwind(rl, rr, vel);
        if (TVD && (g.flag[c] & F_TCX))
            val += psi_surface(rho[c - 2], rl, rr, rho[c + 1], at(g.x.d, i - 2), at(g.x.d, i - 1),
                               at(g.x.d, i), at(g.x.d, i + 1), vel) * (rr - rl);
        rho_u[c] = val;
    }
    if (i < g.nx && j <= g.ny) {
        const double vel = v[c], rb = rho[c - P], rt = rho[c];
        double val = upwind(rb, rt, vel);
        if (TVD && (g.flag[c] & F_TCY))
            val += psi_surface(rho[c - 2 * P], rb, rt, rho[c + P], at(g.y.d, j - 2), at(g.y.d, j - 1),
                               at(g.y.d, j), at(g.y.d, j + 1), vel) * (rt - rb);
        rho_v[c] = val;
    }
}

// ------------------------------------------------------- explicit terms

// T^explicit of cell (i,j), Eq. pl31_1, all inputs at level n-1.
template <bool TVD>
__device__ double explicit_T(const Geo &g, const Level &L, const double *rho_u, const double *rho_v,
                             int c, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const double *T = L.T;
    const double Tp = T[c];
    const double Tw = seen(T, fl, c, c - 1, F_WALL), Te = seen(T, fl, c, c + 1, F_WALL);
    const double Ts = seen(T, fl, c, c - P, F_WALL), Tn = seen(T, fl, c, c + P, F_WALL);
    const double uw = L.u[c], ue = L.u[c + 1], vs = L.v[c], vn = L.v[c + P];
    const double Fw = rho_u[c] * uw * dyj, Fe = rho_u[c + 1] * ue * dyj;
    const double Fs = rho_v[c] * vs * dxi, Fn = rho_v[c + P] * vn * dxi;
    double pw = 0.0, pe = 0.0, ps = 0.0, pn = 0.0;
    if (TVD) {
        if (fl[c + 1] & F_TCX)
            pe = psi_surface(T[c - 1], Tp, Te, T[c + 2], at(g.x.d, i - 1), dxi, at(g.x.d, i + 1), at(g.x.d, i + 2), ue);
        if (fl[c] & F_TCX)
            pw = psi_surface(T[c - 2], Tw, Tp, Te, at(g.x.d, i - 2), at(g.x.d, i - 1), dxi, at(g.x.d, i + 1), uw);
        if (fl[c + P] & F_TCY)
            pn = psi_surface(T[c - P], Tp, Tn, T[c + 2 * P], at(g.y.d, j - 1), dyj, at(g.y.d, j + 1), at(g.y.d, j + 2), vn);
        if (fl[c] & F_TCY)
            ps = psi_surface(T[c - 2 * P], Ts, Tp, Tn, at(g.y.d, j - 2), at(g.y.d, j - 1), dyj, at(g.y.d, j + 1), vs);
    }
    return -Fe * (upwind(Tp, Te, ue) + (Te - Tp) * pe) + Fw * (upwind(Tw, Tp, uw) + (Tp - Tw) * pw)
           - Fn * (upwind(Tp, Tn, vn) + (Tn - Tp) * pn) + Fs * (upwind(Ts, Tp, vs) + (Tp - Ts) * ps);
}

// v^explicit of v face (i,j), Eq. pl15_11, level n-1.
template <bool TVD>
__device__ double explicit_v(const Geo &g, const Level &L, const double *rho_u, int b, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *v = L.v, *u = L.u;
    const double dxi = at(g.x.d, i), dys = at(g.y.d, j - 1), dyp = at(g.y.d, j);
    const double vP = v[b], vW = seen(v, fl, b, b - 1, F_VWALL), vE = seen(v, fl, b, b + 1, F_VWALL);
    const double vS = v[b - P], vN = v[b + P];
    const double uw1 = u[b - P], uw2 = u[b], ue1 = u[b + 1 - P], ue2 = u[b + 1];
    const double Fw1 = rho_u[b - P] * uw1 * dys, Fw2 = rho_u[b] * uw2 * dyp;
    const double Fe1 = rho_u[b + 1 - P] * ue1 * dys, Fe2 = rho_u[b + 1] * ue2 * dyp;
    const double vbs = 0.5 * (vS + vP), vbn = 0.5 * (vP + vN);
    double pw1 = 0, pw2 = 0, pe1 = 0, pe2 = 0, ps = 0, pn = 0;
    if (TVD) {
        if (fl[b + 1] & F_TVX) {
            const double f1 = v[b - 1], f4 = v[b + 2];
            const double d1 = at(g.x.d, i - 1), d3 = at(g.x.d, i + 1), d4 = at(g.x.d, i + 2);
            pe1 = psi_surface(f1, vP, vE, f4, d1, dxi, d3, d4, ue1);
            pe2 = psi_surface(f1, vP, vE, f4, d1, dxi, d3, d4, ue2);
        }
        if (fl[b] & F_TVX) {
            const double f1 = v[b - 2];
            const double d1 = at(g.x.d, i - 2), d2 = at(g.x.d, i - 1), d4 = at(g.x.d, i + 1);
            pw1 = psi_surface(f1, vW, vP, vE, d1, d2, dxi, d4, uw1);
            pw2 = psi_surface(f1, vW, vP, vE, d1, d2, dxi, d4, uw2);
        }
        if (fl[b + P] & F_TVY)
            pn = psi_centre(vS, vP, vN, v[b + 2 * P], dys, dyp, at(g.y.d, j + 1), vbn);
        if (fl[b] & F_TVY)
            ps = psi_centre(v[b - 2 * P], vS, vP, vN, at(g.y.d, j - 2), dys, dyp, vbs);
    }
    return -0.5 * (Fe1 * (upwind(vP, vE, ue1) + (vE - vP) * pe1) + Fe2 * (upwind(vP, vE, ue2) + (vE - vP) * pe2))
           + 0.5 * (Fw1 * (upwind(vW, vP, uw1) + (vP - vW) * pw1) + Fw2 * (upwind(vW, vP, uw2) + (vP - vW) * pw2))
           - dxi * L.rho[b] * vbn * (upwind(vP, vN, vbn) + (vN - vP) * pn)
           + dxi * L.rho[b - P] * vbs * (upwind(vS, vP, vbs) + (vP - vS) * ps);
}

// u^explicit of u face (i,j): the mirror image of Eq. pl15_11, level n-1.
template <bool TVD>
__device__ double explicit_u(const Geo &g, const Level &L, const double *rho_v, int a, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *u = L.u, *v = L.v;
    const double dyj = at(g.y.d, j), dxw = at(g.x.d, i - 1), dxp = at(g.x.d, i);
    const double uP = u[a], uS = seen(u, fl, a, a - P, F_UWALL), uN = seen(u, fl, a, a + P, F_UWALL);
    const double uW = u[a - 1], uE = u[a + 1];
    const double vs1 = v[a - 1], vs2 = v[a], vn1 = v[a - 1 + P], vn2 = v[a + P];
    const double Fs1 = rho_v[a - 1] * vs1 * dxw, Fs2 = rho_v[a] * vs2 * dxp;
    const double Fn1 = rho_v[a - 1 + P] * vn1 * dxw, Fn2 = rho_v[a + P] * vn2 * dxp;
    const double ubw = 0.5 * (uW + uP), ube = 0.5 * (uP + uE);
    double pn1 = 0, pn2 = 0, ps1 = 0, ps2 = 0, pe = 0, pw = 0;
    if (TVD) {
        if (fl[a + P] & F_TUY) {
            const double f1 = u[a - P], f4 = u[a + 2 * P];
            const double d1 = at(g.y.d, j - 1), d3 = at(g.y.d, j + 1), d4 = at(g.y.d, j + 2);
            pn1 = psi_surface(f1, uP, uN, f4, d1, dyj, d3, d4, vn1);
            pn2 = psi_surface(f1, uP, uN, f4, d1, dyj, d3, d4, vn2);
        }
        if (fl[a] & F_TUY) {
            const double f1 = u[a - 2 * P];
            const double d1 = at(g.y.d, j - 2), d2 = at(g.y.d, j - 1), d4 = at(g.y.d, j + 1);
            ps1 = psi_surface(f1, uS, uP, uN, d1, d2, dyj, d4, vs1);
            ps2 = psi_surface(f1, uS, uP, uN, d1, d2, dyj, d4, vs2);
        }
        if (fl[a + 1] & F_TUX)
            pe = psi_centre(uW, uP, uE, u[a + 2], dxw, dxp, at(g.x.d, i + 1), ube);
        if (fl[a] & F_TUX)
            pw = psi_centre(u[a - 2], uW, uP, uE, at(g.x.d, i - 2), dxw, dxp, ubw);
    }
    return -0.5 * (Fn1 * (upwind(uP, uN, vn1) + (uN - uP) * pn1) + Fn2 * (upwind(uP, uN, vn2) + (uN - uP) * pn2))
           + 0.5 * (Fs1 * (upwind(uS, uP, vs1) + (uP - uS) * ps1) + Fs2 * (upwind(uS, uP, vs2) + (uP - uS) * ps2))
           - dyj * L.rho[a] * ube * (upwind(uP, uE, ube) + (uE - uP) * pe)
           + dyj * L.rho[a - 1] * ubw * (upwind(uW, uP, ubw) + (uP - uW) * pw);
}

template <bool TVD>
__global__ void __launch_bounds__(BX *BY) k_explicit_terms(Geo g, Level prev, Work w)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int c = Ix{g.pitch}(i, j);
    if (i > g.nx || j > g.ny) return;
    const uint16_t f = g.flag[c];
    if (i < g.nx && j < g.ny)
        w.Texp[c] = (f & F_FLUID) ? explicit_T<TVD>(g, prev, w.rho_u, w.rho_v, c, i, j) : 0.0;
    if (j < g.ny)
        w.uexp[c] = (f & F_UACT) ? explicit_u<TVD>(g, prev, w.rho_v, c, i, j) : 0.0;
    if (i < g.nx)
        w.vexp[c] = (f & F_VACT) ? explicit_v<TVD>(g, prev, w.rho_u, c, i, j) : 0.0;
}

// ------------------------------------------------------------ temperature

// Energy source S^T_c of cell (i,j), Eq. pl29 with S^T_p = 0 (Eq. pl28):
// viscous dissipation (Eq. pl7) and pressure work; velocities off their
// nodes are bilinear interpolations, reflected across walls.
__device__ double energy_source(const Geo &g, const Coef &k, const Level &L, int c, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *u = L.u, *v = L.v;
    const double dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const double rdx = at(g.x.rd, i), rdy = at(g.y.rd, j);
    const double dudx = (u[c + 1] - u[c]) * rdx;
    const double dvdy = (v[c + P] - v[c]) * rdy;
    const double xl0 = at(g.x.wlo, i), xh0 = at(g.x.whi, i), xl1 = at(g.x.wlo, i + 1), xh1 = at(g.x.whi, i + 1);
    const double yl0 = at(g.y.wlo, j), yh0 = at(g.y.whi, j), yl1 = at(g.y.wlo, j + 1), yh1 = at(g.y.whi, j + 1);
    // v at (x^f_i, y^v_j) and (x^f_{i+1}, y^v_j)
    const double v_w = 0.5 * ((xl0 * seen(v, fl, c, c - 1, F_VWALL) + xh0 * v[c])
                              + (xl0 * seen(v, fl, c + P, c + P - 1, F_VWALL) + xh0 * v[c + P]));
    const double v_e = 0.5 * ((xl1 * v[c] + xh1 * seen(v, fl, c, c + 1, F_VWALL))
                              + (xl1 * v[c + P] + xh1 * seen(v, fl, c + P, c + P + 1, F_VWALL)));
    // u at (x^v_i, y^f_j) and (x^v_i, y^f_{j+1})
    const double u_s = 0.5 * ((yl0 * seen(u, fl, c, c - P, F_UWALL) + yh0 * u[c])
                              + (yl0 * seen(u, fl, c + 1, c + 1 - P, F_UWALL) + yh0 * u[c + 1]));
    const double u_n = 0.5 * ((yl1 * u[c] + yh1 * seen(u, fl, c, c + P, F_UWALL))
                              + (yl1 * u[c + 1] + yh1 * seen(u, fl, c + 1, c + 1 + P, F_UWALL)));
    const double dvdx = (v_e - v_w) * rdx, dudy = (u_n - u_s) * rdy;
    const double div = dudx + dvdy, shear = dvdx + dudy;
    const double phi = 2.0 * (dudx * dudx + dvdy * dvdy) + shear * shear - (2.0 / 3.0) * div * div;
    const double vol = dxi * dyj;
    return (k.CT2f * L.gam[c] * phi + k.CT3f * L.p[c] * div) * vol;
}

// New temperature of fluid cell (i,j): Eq. pl30 with the implicit
// coefficients of Eq. pl31 or the explicit ones of Eq. pl31_1, conductances
// Eq. pl32 with the harmonic mean Eq. pl33.
template <bool IMPL, bool TVD>
__device__ double temperature(const Geo &g, const Coef &k, const Level &prev, const Level &old,
                              const Work &w, int c, int i, int j)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *T = old.T, *gam = old.gam;
    const double dxi = at(g.x.d, i), dyj = at(g.y.d, j);
    const double dxw = at(g.x.d, i - 1), dxe = at(g.x.d, i + 1), dys = at(g.y.d, j - 1), dyn = at(g.y.d, j + 1);
    const double Tp = T[c];
    const double Tw = seen(T, fl, c, c - 1, F_WALL), Te = seen(T, fl, c, c + 1, F_WALL);
    const double Ts = seen(T, fl, c, c - P, F_WALL), Tn = seen(T, fl, c, c + P, F_WALL);
    const double uw = old.u[c], ue = old.u[c + 1], vs = old.v[c], vn = old.v[c + P];
    const double Fw = w.rho_u[c] * uw * dyj, Fe = w.rho_u[c + 1] * ue * dyj;
    const double Fs = w.rho_v[c] * vs * dxi, Fn = w.rho_v[c + P] * vn * dxi;
    const double gp = gam[c];
    const double Dw = k.CT1f * harmonic(gam[c - 1], gp, dxw, dxi) * dyj * at(g.x.rc, i);
    const double De = k.CT1f * harmonic(gp, gam[c + 1], dxi, dxe) * dyj * at(g.x.rc, i + 1);
    const double Ds = k.CT1f * harmonic(gam[c - P], gp, dys, dyj) * dxi * at(g.y.rc, j);
    const double Dn = k.CT1f * harmonic(gp, gam[c + P], dyj, dyn) * dxi * at(g.y.rc, j + 1);
    const double vol = dxi * dyj;
    double a1, a2, a3, a4, a0, texp;
    if (IMPL) {
        double pw = 0.0, pe = 0.0, ps = 0.0, pn = 0.0;
        if (TVD) {
            if (fl[c] & F_TCX)
                pw = psi_surface(T[c - 2], Tw, Tp, Te, at(g.x.d, i - 2), dxw, dxi, dxe, uw);
            if (fl[c + 1] & F_TCX)
                pe = psi_surface(Tw, Tp, Te, T[c + 2], dxw, dxi, dxe, at(g.x.d, i + 2), ue);
            if (fl[c] & F_TCY)
                ps = psi_surface(T[c - 2 * P], Ts, Tp, Tn, at(g.y.d, j - 2), dys, dyj, dyn, vs);
            if (fl[c + P] & F_TCY)
                pn = psi_surface(Ts, Tp, Tn, T[c + 2 * P], dys, dyj, dyn, at(g.y.d, j + 2), vn);
        }
        a1 = pos(Fw) - Fw * pw + Dw;
        a2 = pos(-Fe) - Fe * pe + De;
        a3 = pos(Fs) - Fs * ps + Ds;
        a4 = pos(-Fn) - Fn * pn + Dn;
        a0 = k.dt * (a1 + a2 + a3 + a4 + Fe - Fw + Fn - Fs) + old.rho[c] * vol;
        texp = 0.0;
    } else {
        a1 = Dw; a2 = De; a3 = Ds; a4 = Dn;
        a0 = k.dt * (a1 + a2 + a3 + a4) + old.rho[c] * vol;
        texp = w.Texp[c];
    }
    const double sc = energy_source(g, k, old, c, i, j);
    const double rhs = k.dt * (a1 * Tw + a2 * Te + a3 * Ts + a4 * Tn + sc + texp) + prev.rho[c] * prev.T[c] * vol;
    return rhs / a0;
}

// ------------------------------------------------------ pseudo velocities

// u^ and d^u of u face (i,j) between fluid cells: the mirror image of
// Eqs. pl14-pl16 and pl20 (the 4/3 normal-stress factor on the x direction).
template <bool IMPL, bool TVD>
__device__ void pseudo_u(const Geo &g, const Coef &k, const Level &prev, const Level &old, const Work &w,
                         int a, int i, int j, double &uhat, double &du)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *u = old.u, *v = old.v, *gam = old.gam, *rho = old.rho;
    const double dxw = at(g.x.d, i - 1), dxp = at(g.x.d, i), dyj = at(g.y.d, j);
    const double uP = u[a];
    const double uW = seen(u, fl, a, a - 1, F_UWALL), uE = seen(u, fl, a, a + 1, F_UWALL);
    const double uS = seen(u, fl, a, a - P, F_UWALL), uN = seen(u, fl, a, a + P, F_UWALL);
    const double ubw = 0.5 * (uW + uP), ube = 0.5 * (uP + uE);
    const double Fbw = ubw * rho[a - 1] * dyj, Fbe = ube * rho[a] * dyj;
    const double vs1 = v[a - 1], vs2 = v[a], vn1 = v[a - 1 + P], vn2 = v[a + P];
    const double Fs1 = w.rho_v[a - 1] * vs1 * dxw, Fs2 = w.rho_v[a] * vs2 * dxp;
    const double Fn1 = w.rho_v[a - 1 + P] * vn1 * dxw, Fn2 = w.rho_v[a + P] * vn2 * dxp;
    const double gcs = gamma_corner(g, gam, a, i, j), gcn = gamma_corner(g, gam, a + P, i, j + 1);
    const double Dxw = k.B * gam[a - 1] * dyj * at(g.x.rd, i - 1);
    const double Dxe = k.B * gam[a] * dyj * at(g.x.rd, i);
    const double wsum = dxp + dxw;
    const double Dys = k.B * gcs * wsum * (0.5 * at(g.y.rc, j));
    const double Dyn = k.B * gcn * wsum * (0.5 * at(g.y.rc, j + 1));
    const double r2dt = 0.5 / k.dt;
    const double trans = (rho[a] * dxp + rho[a - 1] * dxw) * dyj * r2dt;
    const double b = (prev.rho[a] * dxp + prev.rho[a - 1] * dxw) * dyj * r2dt * prev.u[a]
                     + k.B * (gcn * (vn2 - vn1) - gcs * (vs2 - vs1)
                              - (2.0 / 3.0) * gam[a] * (vn2 - vs2) + (2.0 / 3.0) * gam[a - 1] * (vn1 - vs1))
                     + k.gx * (rho[a] * dxp + rho[a - 1] * dxw) * dyj * 0.5;
    double a1, a2, a3, a4, a0, uexp;
    if (IMPL) {
        double pw = 0, pe = 0, ps1 = 0, ps2 = 0, pn1 = 0, pn2 = 0;
        if (TVD) {
            if (fl[a] & F_TUX)
                pw = psi_centre(u[a - 2], uW, uP, uE, at(g.x.d, i - 2), dxw, dxp, ubw);
            if (fl[a + 1] & F_TUX)
                pe = psi_centre(uW, uP, uE, u[a + 2], dxw, dxp, at(g.x.d, i + 1), ube);
            if (fl[a] & F_TUY) {
                const double f1 = u[a - 2 * P];
                const double d1 = at(g.y.d, j - 2), d2 = at(g.y.d, j - 1), d4 = at(g.y.d, j + 1);
                ps1 = psi_surface(f1, uS, uP, uN, d1, d2, dyj, d4, vs1);
                ps2 = psi_surface(f1, uS, uP, uN, d1, d2, dyj, d4, vs2);
            }
            if (fl[a + P] & F_TUY) {
                const double f4 = u[a + 2 * P];
                const double d1 = at(g.y.d, j - 1), d3 = at(g.y.d, j + 1), d4 = at(g.y.d, j + 2);
                pn1 = psi_surface(uS, uP, uN, f4, d1, dyj, d3, d4, vn1);
                pn2 = psi_surface(uS, uP, uN, f4, d1, dyj, d3, d4, vn2);
            }
        }
        a1 = pos(Fbw) - Fbw * pw + (4.0 / 3.0) * Dxw;
        a2 = pos(-Fbe) - Fbe * pe + (4.0 / 3.0) * Dxe;
        a3 = 0.5 * (pos(Fs1) - Fs1 * ps1 + pos(Fs2) - Fs2 * ps2) + Dys;
        a4 = 0.5 * (pos(-Fn1) - Fn1 * pn1 + pos(-Fn2) - Fn2 * pn2) + Dyn;
        a0 = a1 + a2 + a3 + a4 + 0.5 * (Fn2 - Fs2 + Fn1 - Fs1) + Fbe - Fbw + trans;
        uexp = 0.0;
    } else {
        a1 = (4.0 / 3.0) * Dxw; a2 = (4.0 / 3.0) * Dxe; a3 = Dys; a4 = Dyn;
        a0 = a1 + a2 + a3 + a4 + trans;
        uexp = w.uexp[a];
    }
    const double r = 1.0 / a0;
    uhat = (a1 * uW + a2 * uE + a3 * uS + a4 * uN + b + uexp) * r;
    du = k.A * dyj * r;
}

// v^ and d^v of v face (i,j) between fluid cells, Eqs. pl14-pl16, pl21
// (implicit, Eq. pl15; explicit, Eq. pl15_11).
template <bool IMPL, bool TVD>
__device__ void pseudo_v(const Geo &g, const Coef &k, const Level &prev, const Level &old, const Work &w,
                         int b, int i, int j, double &vhat, double &dv)
{
    const int P = g.pitch;
    const uint16_t *fl = g.flag;
    const double *u = old.u, *v = old.v, *gam = old.gam, *rho = old.rho;
    const double dys = at(g.y.d, j - 1), dyp = at(g.y.d, j), dxi = at(g.x.d, i);
    const double vP = v[b];
    const double vW = seen(v, fl, b, b - 1, F_VWALL), vE = seen(v, fl, b, b + 1, F_VWALL);
    const double vS = seen(v, fl, b, b - P, F_VWALL), vN = seen(v, fl, b, b + P, F_VWALL);
    const double vbs = 0.5 * (vS + vP), vbn = 0.5 * (vP + vN);
    const double Fbs = vbs * rho[b - P] * dxi, Fbn = vbn * rho[b] * dxi;
    const double uw1 = u[b - P], uw2 = u[b], ue1 = u[b + 1 - P], ue2 = u[b + 1];
    const double Fw1 = w.rho_u[b - P] * uw1 * dys, Fw2 = w.rho_u[b] * uw2 * dyp;
    const double Fe1 = w.rho_u[b + 1 - P] * ue1 * dys, Fe2 = w.rho_u[b + 1] * ue2 * dyp;
    const double gcw = gamma_corner(g, gam, b, i, j), gce = gamma_corner(g, gam, b + 1, i + 1, j);
    const double hsum = dyp + dys;
    const double Dxw = k.B * gcw * hsum * (0.5 * at(g.x.rc, i));
    const double Dxe = k.B * gce * hsum * (0.5 * at(g.x.rc, i + 1));
    const double Dys = k.B * gam[b - P] * dxi * at(g.y.rd, j - 1);
    const double Dyn = k.B * gam[b] * dxi * at(g.y.rd, j);
    const double r2dt = 0.5 / k.dt;
    const double trans = (rho[b] * dyp + rho[b - P] * dys) * dxi * r2dt;
    const double bsrc = (prev.rho[b] * dyp + prev.rho[b - P] * dys) * dxi * r2dt * prev.v[b]
                        + k.B * (gce * (ue2 - ue1) - gcw * (uw2 - uw1)
                                 - (2.0 / 3.0) * gam[b] * (ue2 - uw2) + (2.0 / 3.0) * gam[b - P] * (ue1 - uw1))
                        + k.gy * (rho[b] * dyp + rho[b - P] * dys) * dxi * 0.5;
    double a1, a2, a3, a4, a0, vexp;
    if (IMPL) {
        double pw1 = 0, pw2 = 0, pe1 = 0, pe2 = 0, ps = 0, pn = 0;
        if (TVD) {
            if (fl[b] & F_TVX) {
                const double f1 = v[b - 2];
                const double d1 = at(g.x.d, i - 2), d2 = at(g.x.d, i - 1), d4 = at(g.x.d, i + 1);
                pw1 = psi_surface(f1, vW, vP, vE, d1, d2, dxi, d4, uw1);
                pw2 = psi_surface(f1, vW, vP, vE, d1, d2, dxi, d4, uw2);
            }
            if (fl[b + 1] & F_TVX) {
                const double f4 = v[b + 2];
                const double d1 = at(g.x.d, i - 1), d3 = at(g.x.d, i + 1), d4 = at(g.x.d, i + 2);
                pe1 = psi_surface(vW, vP, vE, f4, d1, dxi, d3, d4, ue1);
                pe2 = psi_surface(vW, vP, vE, f4, d1, dxi, d3, d4, ue2);
            }
            if (fl[b] & F_TVY)
                ps = psi_centre(v[b - 2 * P], vS, vP, vN, at(g.y.d, j - 2), dys, dyp, vbs);
            if (fl[b + P] & F_TVY)
                pn = psi_centre(vS, vP, vN, v[b + 2 * P], dys, dyp, at(g.y.d, j + 1), vbn);
        }
        a1 = 0.5 * (pos(Fw2) - Fw2 * pw2 + pos(Fw1) - Fw1 * pw1) + Dxw;
        a2 = 0.5 * (pos(-Fe2) - Fe2 * pe2 + pos(-Fe1) - Fe1 * pe1) + Dxe;
        a3 = pos(Fbs) - Fbs * ps + (4.0 / 3.0) * Dys;
        a4 = pos(-Fbn) - Fbn * pn + (4.0 / 3.0) * Dyn;
        a0 = a1 + a2 + a3 + a4 + 0.5 * (Fe2 - Fw2 + Fe1 - Fw1) + Fbn - Fbs + trans;
        vexp = 0.0;
    } else {
        a1 = Dxw; a2 = Dxe; a3 = (4.0 / 3.0) * Dys; a4 = (4.0 / 3.0) * Dyn;
        a0 = a1 + a2 + a3 + a4 + trans;
        vexp = w.vexp[b];
    }
    const double r = 1.0 / a0;
    vhat = (a1 * vW + a2 * vE + a3 * vS + a4 * vN + bsrc + vexp) * r;
    dv = k.A * dxi * r;
}

template <bool IMPL, bool TVD>
__global__ void __launch_bounds__(BX *BY) k_assemble(Geo g, Coef k, Level prev, Level old, Level nw, Work w)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i > g.nx || j > g.ny) return;
    const int c = Ix{g.pitch}(i, j);
    const uint16_t f = g.flag[c];
    if (i < g.nx && j < g.ny && (f & F_FLUID))
        nw.T[c] = temperature<IMPL, TVD>(g, k, prev, old, w, c, i, j);
    if (j < g.ny) {
        double uh = old.u[c], d = 0.0;        // faces that are not unknowns: stored u, d = 0
        if (f & F_UACT)
            pseudo_u<IMPL, TVD>(g, k, prev, old, w, c, i, j, uh, d);
        w.uhat[c] = uh;
        w.du[c] = d;
    }
    if (i < g.nx) {
        double vh = old.v[c], d = 0.0;
        if (f & F_VACT)
            pseudo_v<IMPL, TVD>(g, k, prev, old, w, c, i, j, vh, d);
        w.vhat[c] = vh;
        w.dv[c] = d;
    }
}

// ---------------------------------------------------------------- pressure

// Eqs. pl23, pl24 with the new T (point Jacobi in p^old), then rho = p/T
// (Eq. pl5) and Gamma = T^omega, with the p and T residual maxima.
__global__ void __launch_bounds__(BX *BY) k_pressure(Geo g, Coef k, Level prev, Level old, Level nw, Work w)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int P = g.pitch;
    unsigned long long rp = 0, rT = 0;
    if (i < g.nx && j < g.ny) {
        const int c = Ix{P}(i, j);
        if (g.flag[c] & F_FLUID) {
            const double dxi = at(g.x.d, i), dyj = at(g.y.d, j);
            const double ru_w = w.rho_u[c], ru_e = w.rho_u[c + 1], rv_s = w.rho_v[c], rv_n = w.rho_v[c + P];
            const double apw = ru_w * w.du[c] * dyj, ape = ru_e * w.du[c + 1] * dyj;
            const double aps = rv_s * w.dv[c] * dxi, apn = rv_n * w.dv[c + P] * dxi;
            const double bpw = ru_w * w.uhat[c] * dyj, bpe = ru_e * w.uhat[c + 1] * dyj;
            const double bps = rv_s * w.vhat[c] * dxi, bpn = rv_n * w.vhat[c + P] * dxi;
            const double Tn = nw.T[c];
            const double vol = dxi * dyj;
            const double ap0 = vol / Tn + (apw + ape + aps + apn) * k.dt;
            const double bp = prev.rho[c] * vol - (bpe - bpw + bpn - bps) * k.dt;
            const double pn = ((apw * old.p[c - 1] + ape * old.p[c + 1] + aps * old.p[c - P] + apn * old.p[c + P]) * k.dt
                               + bp) / ap0;
            nw.p[c] = pn;
            nw.rho[c] = pn / Tn;
            nw.gam[c] = (k.omega == 0.5) ? sqrt(Tn) : pow(Tn, k.omega);
            rp = ordered(pn - old.p[c]);
            rT = ordered(Tn - old.T[c]);
        }
    }
    block_max2(rp, rT, &w.res[2], &w.res[3]);
}

// -------------------------------------------------------------- velocity

// Eqs. pl18, pl19: velocities of the face unknowns from the new pressure.
__global__ void __launch_bounds__(BX *BY) k_velocity(Geo g, Level old, Level nw, Work w)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int P = g.pitch;
    unsigned long long ru = 0, rv = 0;
    if (i <= g.nx && j <= g.ny) {
        const int c = Ix{P}(i, j);
        const uint16_t f = g.flag[c];
        if (j < g.ny && (f & F_UACT)) {
            const double un = w.uhat[c] - w.du[c] * (nw.p[c] - nw.p[c - 1]);
            nw.u[c] = un;
            ru = ordered(un - old.u[c]);
        }
        if (i < g.nx && (f & F_VACT)) {
            const double vn = w.vhat[c] - w.dv[c] * (nw.p[c] - nw.p[c - P]);
            nw.v[c] = vn;
            rv = ordered(vn - old.v[c]);
        }
    }
    block_max2(ru, rv, &w.res[0], &w.res[1]);
}

// ------------------------------------------------------------ ghost copies

// West/east sides, one thread per row j in [0, ny].
__global__ void k_ghost_we(Geo g, Sides s, Level L)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > g.ny) return;
    const Ix ix{g.pitch};
    const int nx = g.nx;
    double *sc[4] = {L.p, L.T, L.rho, L.gam};
    if (s.kind[SIDE_E] == BC_OUTFLOW) {
        if (j < g.ny) {
            const int src = ix(nx - 1, j);
            for (int q = 0; q < 4; q++) {
                sc[q][ix(nx, j)] = sc[q][src];
                sc[q][ix(nx + 1, j)] = sc[q][src];
            }
            const double us = L.u[src];
            L.u[ix(nx, j)] = us;
            L.u[ix(nx + 1, j)] = us;
            L.u[ix(nx + 2, j)] = us;
        }
        const double vs = L.v[ix(nx - 1, j)];
        L.v[ix(nx, j)] = vs;
        L.v[ix(nx + 1, j)] = vs;
    }
    if (s.kind[SIDE_W] == BC_SYMMETRY) {
        if (j < g.ny) {
            for (int q = 0; q < 4; q++) {
                sc[q][ix(-1, j)] = sc[q][ix(0, j)];
                sc[q][ix(-2, j)] = sc[q][ix(1, j)];
            }
            L.u[ix(-1, j)] = -L.u[ix(1, j)];
            L.u[ix(-2, j)] = -L.u[ix(2, j)];
        }
        L.v[ix(-1, j)] = L.v[ix(0, j)];
        L.v[ix(-2, j)] = L.v[ix(1, j)];
    }
    if (s.kind[SIDE_E] == BC_SYMMETRY) {
        if (j < g.ny) {
            for (int q = 0; q < 4; q++) {
                sc[q][ix(nx, j)] = sc[q][ix(nx - 1, j)];
                sc[q][ix(nx + 1, j)] = sc[q][ix(nx - 2, j)];
            }
            L.u[ix(nx + 1, j)] = -L.u[ix(nx - 1, j)];
            L.u[ix(nx + 2, j)] = -L.u[ix(nx - 2, j)];
        }
        L.v[ix(nx, j)] = L.v[ix(nx - 1, j)];
        L.v[ix(nx + 1, j)] = L.v[ix(nx - 2, j)];
    }
}

// South/north symmetry sides, one thread per column i in [-2, nx+2].
__global__ void k_ghost_sn(Geo g, Sides s, Level L)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - G;
    if (i > g.nx + G) return;
    const Ix ix{g.pitch};
    const int ny = g.ny;
    double *sc[4] = {L.p, L.T, L.rho, L.gam};
    const bool cell = i <= g.nx + 1;
    if (s.kind[SIDE_S] == BC_SYMMETRY) {
        if (cell)
            for (int q = 0; q < 4; q++) {
                sc[q][ix(i, -1)] = sc[q][ix(i, 0)];
                sc[q][ix(i, -2)] = sc[q][ix(i, 1)];
            }
        L.u[ix(i, -1)] = L.u[ix(i, 0)];
        L.u[ix(i, -2)] = L.u[ix(i, 1)];
        if (cell) {
            L.v[ix(i, -1)] = -L.v[ix(i, 1)];
            L.v[ix(i, -2)] = -L.v[ix(i, 2)];
        }
    }
    if (s.kind[SIDE_N] == BC_SYMMETRY) {
        if (cell)
            for (int q = 0; q < 4; q++) {
                sc[q][ix(i, ny)] = sc[q][ix(i, ny - 1)];
                sc[q][ix(i, ny + 1)] = sc[q][ix(i, ny - 2)];
            }
        L.u[ix(i, ny)] = L.u[ix(i, ny - 1)];
        L.u[ix(i, ny + 1)] = L.u[ix(i, ny - 2)];
        if (cell) {
            L.v[ix(i, ny + 1)] = -L.v[ix(i, ny - 1)];
            L.v[ix(i, ny + 2)] = -L.v[ix(i, ny - 2)];
        }
    }
}

// ----------------------------------------------------- state maintenance

// rho = p/T and Gamma = T^omega of every fluid cell.
__global__ void k_derive(Geo g, Coef k, Level L)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int c = Ix{g.pitch}(i, j);
    if (!(g.flag[c] & F_FLUID)) return;
    const double T = L.T[c];
    L.rho[c] = L.p[c] / T;
    L.gam[c] = (k.omega == 0.5) ? sqrt(T) : pow(T, k.omega);
}

__device__ __forceinline__ double *field_of(const Level &L, int f)
{
    switch (f) {
    case 0: return L.u;
    case 1: return L.v;
    case 2: return L.p;
    case 3: return L.T;
    case 4: return L.rho;
    default: return L.gam;
    }
}

// Write the unknowns of one field from a logical-shape array.
__global__ void k_scatter(Geo g, int field, const double *src, Level L)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny;
    const int w = field == 0 ? nx + 1 : nx, h = field == 1 ? ny + 1 : ny;
    if (i >= w || j >= h) return;
    const int c = Ix{g.pitch}(i, j);
    const uint16_t f = g.flag[c];
    const uint32_t bit = field == 0 ? F_UACT : field == 1 ? F_VACT : F_FLUID;
    if (f & bit)
        field_of(L, field)[c] = src[(size_t)j * w + i];
}

// Read one field into a logical-shape array (boundary values included).
__global__ void k_gather(Geo g, int field, Level L, double *dst)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny;
    const int w = field == 0 ? nx + 1 : nx, h = field == 1 ? ny + 1 : ny;
    if (i >= w || j >= h) return;
    dst[(size_t)j * w + i] = field_of(L, field)[Ix{g.pitch}(i, j)];
}

dim3 grid_of(const Geo &g)
{
    return dim3((unsigned)((g.nx + 1 + BX - 1) / BX), (unsigned)((g.ny + 1 + BY - 1) / BY));
}

}  // namespace

// ------------------------------------------------------------- launchers

void launch_face_densities(const Geo &g, const Level &lv, const Work &w, bool tvd, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (tvd)
        k_face_densities<true><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, lv.u, lv.v, lv.rho, w.rho_u, w.rho_v);
    else
        k_face_densities<false><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, lv.u, lv.v, lv.rho, w.rho_u, w.rho_v);
}

void launch_explicit_terms(const Geo &g, const Level &prev, const Work &w, bool tvd, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (tvd)
        k_explicit_terms<true><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, prev, w);
    else
        k_explicit_terms<false><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, prev, w);
}

void launch_assemble(const Geo &g, const Coef &c, const Level &prev, const Level &old, const Level &nw,
                     const Work &w, bool implicit, bool tvd, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 gr = grid_of(g), bl(BX, BY);
    if (implicit && tvd) k_assemble<true, true><<<gr, bl, 0, s>>>(g, c, prev, old, nw, w);
    else if (implicit) k_assemble<true, false><<<gr, bl, 0, s>>>(g, c, prev, old, nw, w);
    else if (tvd) k_assemble<false, true><<<gr, bl, 0, s>>>(g, c, prev, old, nw, w);
    else k_assemble<false, false><<<gr, bl, 0, s>>>(g, c, prev, old, nw, w);
}

void launch_pressure(const Geo &g, const Coef &c, const Level &prev, const Level &old, const Level &nw,
                     const Work &w, void *stream)
{
    k_pressure<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, c, prev, old, nw, w);
}

void launch_velocity(const Geo &g, const Level &old, const Level &nw, const Work &w, void *stream)
{
    k_velocity<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, old, nw, w);
}

void launch_ghosts(const Geo &g, const Sides &sd, const Level &lv, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const bool we = sd.kind[SIDE_E] == BC_OUTFLOW || sd.kind[SIDE_E] == BC_SYMMETRY || sd.kind[SIDE_W] == BC_SYMMETRY;
    const bool sn = sd.kind[SIDE_S] == BC_SYMMETRY || sd.kind[SIDE_N] == BC_SYMMETRY;
    if (we)
        k_ghost_we<<<(g.ny + 1 + 127) / 128, 128, 0, s>>>(g, sd, lv);
    if (sn)
        k_ghost_sn<<<(g.nx + 2 * G + 1 + 127) / 128, 128, 0, s>>>(g, sd, lv);
}

void launch_derive(const Geo &g, const Coef &c, const Level &lv, void *stream)
{
    k_derive<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, c, lv);
}

void launch_scatter(const Geo &g, int field, const double *src, const Level &lv, void *stream)
{
    k_scatter<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, field, src, lv);
}

void launch_gather(const Geo &g, int field, const Level &lv, double *dst, void *stream)
{
    k_gather<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, field, lv, dst);
}

}  // namespace stg
