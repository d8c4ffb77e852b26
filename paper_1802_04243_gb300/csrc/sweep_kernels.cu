// sweep_kernels.cu -- CUDA kernels of one SIMPLE-TS time step
// (K. S. Shterev, arXiv:1802.04243, Sections 3.1 and 3.2) for sm_103a.
// The equation kernels are templated on the arithmetic type: double for the
// FP64 path, float for the FP32 assembly of the mixed-precision path (whose
// pressure accumulation, equation of state and residuals stay FP64), and
// df64 (double-float, df64.cuh) for the DF64 path, which runs the whole
// iteration on the FP32 pipe.
//
// One loop-2 iteration (Section 3.1, Figs. 1 and 2, GPU column) runs as
//   k_faces      rho^u, rho^v, mass fluxes and conductivities of every face (Eqs. pl8-pl11, pl33)
//   k_assemble   T, u^/d^u, v^/d^v of every node         (Eqs. pl14-pl16, pl20, pl21, pl28-pl33)
//   k_pressure   p, rho = p/T, Gamma = T^omega, |dp|, |dT| (Eqs. pl23, pl24, pl5)
//   k_velocity   u, v from the new p, |du|, |dv|          (Eqs. pl18, pl19)
//   k_ghost_*    outflow / symmetry ghost copies
// and, once per step for the explicit scheme, k_explicit (Eqs. pl15_11,
// pl31_1 and the u mirror).  Each thread owns one grid position (i, j) and
// the cell, the u face and the v face with that index; the equation kernels
// walk a list of tiles of one or more problems.  This file holds the ghost,
// conversion, gather/scatter and check kernels and the launchers; the
// equation kernels are in phase_kernels.cuh, compiled once per arithmetic.
//
// Boundary rules: wall ghost and obstacle cells hold the wall state; a
// temperature or tangential velocity read across a wall is reflected about
// the value at the wall surface (2 phi_s - phi_reader): the wall value, or
// with velocity slip / temperature jump the value of Eqs. pl38, pl39 (seen_s);
// TVD corrections apply only where the flag of the face says all four stencil
// nodes are unknowns.
#include "sweep_bodies.cuh"

namespace stg {
namespace {

// ------------------------------------------------------------ ghost copies

// West/east sides, one thread per row j in [0, ny].
template <typename R>
__global__ void k_ghost_we(GeoT<R> g, Sides s, LevelT<R> L)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > g.ny) return;
    const Ix ix{g.pitch};
    const int nx = g.nx;
    R *sc[4] = {L.p, L.T, L.rho, L.gam};
    if (s.kind[SIDE_E] == BC_OUTFLOW) {
        if (j < g.ny) {
            const int src = ix(nx - 1, j);
            for (int q = 0; q < 4; q++) {
                sc[q][ix(nx, j)] = sc[q][src];
                sc[q][ix(nx + 1, j)] = sc[q][src];
            }
            const R us = L.u[src];
            L.u[ix(nx, j)] = us;
            L.u[ix(nx + 1, j)] = us;
            L.u[ix(nx + 2, j)] = us;
        }
        const R vs = L.v[ix(nx - 1, j)];
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
template <typename R>
__global__ void k_ghost_sn(GeoT<R> g, Sides s, LevelT<R> L)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) + (s.col1 > 0 ? s.col0 : -G);
    if (i > g.nx + G || (s.col1 > 0 && i >= s.col1)) return;
    const Ix ix{g.pitch};
    const int ny = g.ny;
    R *sc[4] = {L.p, L.T, L.rho, L.gam};
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

// FP32 shadow copy of a whole FP64 level (every element, ghosts included).
__global__ void k_shadow(Level L, LevelT<float> S, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        S.u[q] = (float)L.u[q];
        S.v[q] = (float)L.v[q];
        S.p[q] = (float)L.p[q];
        S.T[q] = (float)L.T[q];
        S.rho[q] = (float)L.rho[q];
        S.gam[q] = (float)L.gam[q];
    }
}


// Whole-level conversions FP64 <-> double-float, ghosts included.
__global__ void k_split(Level L, LevelT<df64> D, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        D.u[q] = dfl::split_dev(L.u[q]);
        D.v[q] = dfl::split_dev(L.v[q]);
        D.p[q] = dfl::split_dev(L.p[q]);
        D.T[q] = dfl::split_dev(L.T[q]);
        D.rho[q] = dfl::split_dev(L.rho[q]);
        D.gam[q] = dfl::split_dev(L.gam[q]);
    }
}

__global__ void k_join(LevelT<df64> D, Level L, size_t n)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        L.u[q] = dfl::join(D.u[q]);
        L.v[q] = dfl::join(D.v[q]);
        L.p[q] = dfl::join(D.p[q]);
        L.T[q] = dfl::join(D.T[q]);
        L.rho[q] = dfl::join(D.rho[q]);
        L.gam[q] = dfl::join(D.gam[q]);
    }
}

// ----------------------------------------------------- state maintenance

// rho = p/T and Gamma = T^omega of every fluid cell, evaluated exactly as
// the pressure kernel evaluates them (so a state written out and set again
// continues bit for bit).
__global__ void k_derive(Geo g, Coef k, Level L, int i0, int i1)
{
    const int i = i0 + blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= i1 || i >= g.nx || j >= g.ny) return;
    const int c = Ix{g.pitch}(i, j);
    if (!(g.flag[c] & F_FLUID)) return;
    const double T = L.T[c];
    L.rho[c] = L.p[c] * recip(T);
    L.gam[c] = gamma_of(T, k.omega);
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

// Read one field into a logical-shape array (boundary values included), the
// columns [i0, i1) of it.
__global__ void k_gather(Geo g, int field, Level L, double *dst, int i0, int i1)
{
    const int i = i0 + blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny;
    const int w = field == 0 ? nx + 1 : nx, h = field == 1 ? ny + 1 : ny;
    if (i >= w || i >= i1 || j >= h) return;
    dst[(size_t)j * w + i] = field_of(L, field)[Ix{g.pitch}(i, j)];
}

// FP64 view of a mixed-precision level over columns [i0, i1) (widen_mixed_at).
__global__ void k_widen_mixed(Geo g, Level L, LevelT<float> S, int east_outflow, int i0, int i1)
{
    const int i = i0 + blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= i1) return;
    widen_mixed_at(g, L, S, east_outflow, i, j);
}

// One 4-byte word of each halo block per thread; blockIdx.y picks the block.
__global__ void k_halo_copies(const HaloCopy *copies, int n)
{
    const HaloCopy c = copies[blockIdx.y];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= c.words * c.rows) return;
    const int r = q / c.words, x = q - r * c.words;
    c.dst[(size_t)r * c.dpitch + x] = c.src[(size_t)r * c.spitch + x];
}

// All four fields of a staged state (u, v, p, T back to back in their
// logical shapes) into the unknowns of a level, with rho and Gamma derived
// as k_derive derives them; one thread per position.
__global__ void k_scatter_state(Geo g, Coef k, const double *st, Level L)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny;
    if (i > nx || j > ny) return;
    const size_t nu = (size_t)(nx + 1) * ny, nv = (size_t)nx * (ny + 1), nc = (size_t)nx * ny;
    const int c = Ix{g.pitch}(i, j);
    const uint16_t f = g.flag[c];
    if (j < ny && (f & F_UACT)) L.u[c] = st[(size_t)j * (nx + 1) + i];
    if (i < nx && (f & F_VACT)) L.v[c] = st[nu + (size_t)j * nx + i];
    if (i < nx && j < ny && (f & F_FLUID)) {
        const size_t q = (size_t)j * nx + i;
        const double p = st[nu + nv + q], T = st[nu + nv + nc + q];
        L.p[c] = p;
        L.T[c] = T;
        L.rho[c] = p * recip(T);
        L.gam[c] = gamma_of(T, k.omega);
    }
}

// All four fields of a level into four arrays in their logical shapes
// (device memory, or page-locked host memory the device addresses),
// boundary values included.
__global__ void k_gather_state(Geo g, Level L, StatePtrs dst)
{
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int nx = g.nx, ny = g.ny;
    if (i > nx || j > ny) return;
    const int c = Ix{g.pitch}(i, j);
    if (j < ny) dst.f[0][(size_t)j * (nx + 1) + i] = L.u[c];
    if (i < nx) dst.f[1][(size_t)j * nx + i] = L.v[c];
    if (i < nx && j < ny) {
        const size_t q = (size_t)j * nx + i;
        dst.f[2][q] = L.p[c];
        dst.f[3][q] = L.T[c];
    }
}

// Copy of a state from four arrays the device addresses (u, v, p, T in their
// logical shapes, e.g. page-locked host memory) into the staging array, with
// the admissibility check of k_validate_state.
__global__ void k_stage_state(StateSrc src, size_t nu, size_t nv, size_t nc, double *stage, unsigned *bad)
{
    const size_t n = nu + nv + 2 * nc;
    unsigned b = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        double x;
        if (q < nu) x = src.f[0][q];
        else if (q < nu + nv) x = src.f[1][q - nu];
        else if (q < nu + nv + nc) x = src.f[2][q - nu - nv];
        else x = src.f[3][q - nu - nv - nc];
        stage[q] = x;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
        const bool finite = ((bits >> 52) & 0x7FFull) != 0x7FFull;
        if (!finite || (q >= nu + nv && !positive(x))) b = 1u;
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// recip(x) next to the IEEE quotient 1/x, for the check of the reciprocal.
// root(x) next to the IEEE square root of x, for the check of the root.
__global__ void k_sqrt_check(const double *x, double *out, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out[2 * q] = root(x[q]);
    out[2 * q + 1] = sqrt(x[q]);
}

__global__ void k_recip_check(const double *x, double *out, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out[2 * q] = recip(x[q]);
    out[2 * q + 1] = 1.0 / x[q];
}

// Admissibility of a staged state (u, v, p, T back to back): every value
// finite, p and T positive.  Bit tests only.
__global__ void k_validate_state(const double *st, size_t nu, size_t nv, size_t nc, unsigned *bad)
{
    const size_t n = nu + nv + 2 * nc;
    unsigned b = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long x = (unsigned long long)__double_as_longlong(st[q]);
        const bool finite = ((x >> 52) & 0x7FFull) != 0x7FFull;
        const bool need_positive = q >= nu + nv;
        if (!finite || (need_positive && !positive(st[q]))) b = 1u;
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

template <typename R>
dim3 grid_of(const GeoT<R> &g)
{
    return dim3((unsigned)((g.nx + 1 + BX - 1) / BX), (unsigned)((g.ny + 1 + BY - 1) / BY));
}

}  // namespace

// ------------------------------------------------------------- launchers

int ghost_kernels(const Sides &sd, bool after_velocity)
{
    const bool we = (!after_velocity && sd.kind[SIDE_E] == BC_OUTFLOW) || sd.kind[SIDE_E] == BC_SYMMETRY ||
                    sd.kind[SIDE_W] == BC_SYMMETRY;
    const bool sn = sd.kind[SIDE_S] == BC_SYMMETRY || sd.kind[SIDE_N] == BC_SYMMETRY;
    return (int)we + (int)sn;
}

void launch_ghosts(const Geo &g, const Sides &sd, const Level &lv, bool after_velocity, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const bool we = (!after_velocity && sd.kind[SIDE_E] == BC_OUTFLOW) || sd.kind[SIDE_E] == BC_SYMMETRY ||
                    sd.kind[SIDE_W] == BC_SYMMETRY;
    const bool sn = sd.kind[SIDE_S] == BC_SYMMETRY || sd.kind[SIDE_N] == BC_SYMMETRY;
    if (we)
        k_ghost_we<double><<<(g.ny + 1 + 127) / 128, 128, 0, s>>>(g, sd, lv);
    if (sn)
        k_ghost_sn<double><<<(g.nx + 2 * G + 1 + 127) / 128, 128, 0, s>>>(g, sd, lv);
}

void launch_ghosts_f32(const Mixed &m, const Sides &sd, int level, bool after_velocity, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const bool we = (!after_velocity && sd.kind[SIDE_E] == BC_OUTFLOW) || sd.kind[SIDE_E] == BC_SYMMETRY ||
                    sd.kind[SIDE_W] == BC_SYMMETRY;
    const bool sn = sd.kind[SIDE_S] == BC_SYMMETRY || sd.kind[SIDE_N] == BC_SYMMETRY;
    if (we)
        k_ghost_we<float><<<(m.g.ny + 1 + 127) / 128, 128, 0, s>>>(m.g, sd, m.lv[level]);
    if (sn)
        k_ghost_sn<float><<<(m.g.nx + 2 * G + 1 + 127) / 128, 128, 0, s>>>(m.g, sd, m.lv[level]);
}

void launch_ghosts_df(const DoubleFloat &d, const Sides &sd, int level, bool after_velocity, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const bool we = (!after_velocity && sd.kind[SIDE_E] == BC_OUTFLOW) || sd.kind[SIDE_E] == BC_SYMMETRY ||
                    sd.kind[SIDE_W] == BC_SYMMETRY;
    const bool sn = sd.kind[SIDE_S] == BC_SYMMETRY || sd.kind[SIDE_N] == BC_SYMMETRY;
    if (we)
        k_ghost_we<df64><<<(d.g.ny + 1 + 127) / 128, 128, 0, s>>>(d.g, sd, d.lv[level]);
    if (sn)
        k_ghost_sn<df64><<<(d.g.nx + 2 * G + 1 + 127) / 128, 128, 0, s>>>(d.g, sd, d.lv[level]);
}

void launch_split(const Level &lv, const LevelT<df64> &d, size_t nelem, void *stream)
{
    const int blocks = (int)((nelem + 255) / 256 < 4096 ? (nelem + 255) / 256 : 4096);
    k_split<<<blocks, 256, 0, (cudaStream_t)stream>>>(lv, d, nelem);
}

void launch_join(const LevelT<df64> &d, const Level &lv, size_t nelem, void *stream)
{
    const int blocks = (int)((nelem + 255) / 256 < 4096 ? (nelem + 255) / 256 : 4096);
    k_join<<<blocks, 256, 0, (cudaStream_t)stream>>>(d, lv, nelem);
}

void launch_shadow(const Geo &g, const Level &lv, const LevelT<float> &lv32, size_t nelem, void *stream)
{
    (void)g;
    const int blocks = (int)((nelem + 255) / 256 < 4096 ? (nelem + 255) / 256 : 4096);
    k_shadow<<<blocks, 256, 0, (cudaStream_t)stream>>>(lv, lv32, nelem);
}

void launch_sqrt_check(const double *x, double *out, int n, void *stream)
{
    if (n > 0) k_sqrt_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, out, n);
}

void launch_recip_check(const double *x, double *out, int n, void *stream)
{
    if (n > 0) k_recip_check<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(x, out, n);
}

void launch_validate_state(const double *stage, size_t nu, size_t nv, size_t nc, unsigned *bad, void *stream)
{
    const size_t n = nu + nv + 2 * nc;
    const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    k_validate_state<<<blocks, 256, 0, (cudaStream_t)stream>>>(stage, nu, nv, nc, bad);
}

void launch_derive(const Geo &g, const Coef &c, const Level &lv, void *stream)
{
    k_derive<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, c, lv, 0, g.nx);
}

void launch_derive_cols(const Geo &g, const Coef &c, const Level &lv, int i0, int i1, void *stream)
{
    if (i1 <= i0) return;
    const dim3 grid((unsigned)((i1 - i0 + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY));
    k_derive<<<grid, dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, c, lv, i0, i1);
}

void launch_scatter_state(const Geo &g, const Coef &c, const double *stage, const Level &lv, void *stream)
{
    k_scatter_state<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, c, stage, lv);
}

void launch_gather_state(const Geo &g, const Level &lv, const StatePtrs &dst, void *stream)
{
    k_gather_state<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, lv, dst);
}

void launch_stage_state(const StateSrc &src, size_t nu, size_t nv, size_t nc, double *stage, unsigned *bad,
                        void *stream)
{
    const size_t n = nu + nv + 2 * nc;
    const int blocks = (int)((n + 255) / 256 < 2048 ? (n + 255) / 256 : 2048);
    k_stage_state<<<blocks, 256, 0, (cudaStream_t)stream>>>(src, nu, nv, nc, stage, bad);
}

void launch_scatter(const Geo &g, int field, const double *src, const Level &lv, void *stream)
{
    k_scatter<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, field, src, lv);
}

void launch_gather(const Geo &g, int field, const Level &lv, double *dst, void *stream)
{
    k_gather<<<grid_of(g), dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, field, lv, dst, 0, g.nx + 1);
}

void launch_gather_cols(const Geo &g, int field, const Level &lv, double *dst, int i0, int i1, void *stream)
{
    if (i1 <= i0) return;
    const dim3 grid((unsigned)((i1 - i0 + BX - 1) / BX), (unsigned)((g.ny + 1 + BY - 1) / BY));
    k_gather<<<grid, dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, field, lv, dst, i0, i1);
}

void launch_widen_mixed(const Geo &g, const Level &lv, const LevelT<float> &s32, bool east_outflow, int i0, int i1,
                        void *stream)
{
    if (i1 <= i0) return;
    const dim3 grid((unsigned)((i1 - i0 + BX - 1) / BX), (unsigned)((g.ny + 1 + BY - 1) / BY));
    k_widen_mixed<<<grid, dim3(BX, BY), 0, (cudaStream_t)stream>>>(g, lv, s32, east_outflow ? 1 : 0, i0, i1);
}

void launch_halo_copies(const HaloCopy *copies, int n, int max_words, void *stream)
{
    if (n <= 0 || max_words <= 0) return;
    k_halo_copies<<<dim3((unsigned)((max_words + 255) / 256), (unsigned)n), 256, 0, (cudaStream_t)stream>>>(copies, n);
}

// The equation kernels' launchers dispatch to the per-arithmetic
// translation units (phase_fp64.cu, phase_mixed.cu, phase_df64.cu).
void launch_faces(const BatchPlan &bp, int prec, int level, bool tvd, bool limiters, void *stream)
{
    const int lim = tvd && limiters;
    if (prec == PREC_DF64) launch_faces_of<PREC_DF64>(bp, level, tvd, lim, stream);
    else if (prec == PREC_MIXED) launch_faces_of<PREC_MIXED>(bp, level, tvd, lim, stream);
    else launch_faces_of<PREC_FP64>(bp, level, tvd, lim, stream);
}

void launch_explicit(const BatchPlan &bp, int prec, int prev, bool tvd, void *stream)
{
    if (prec == PREC_DF64) launch_explicit_of<PREC_DF64>(bp, prev, tvd, stream);
    else if (prec == PREC_MIXED) launch_explicit_of<PREC_MIXED>(bp, prev, tvd, stream);
    else launch_explicit_of<PREC_FP64>(bp, prev, tvd, stream);
}

void launch_assemble(const BatchPlan &bp, int prec, int prev, int old, int nw, bool implicit, bool tvd,
                     void *stream)
{
    if (prec == PREC_DF64) launch_assemble_of<PREC_DF64>(bp, prev, old, nw, implicit, tvd, stream);
    else if (prec == PREC_MIXED) launch_assemble_of<PREC_MIXED>(bp, prev, old, nw, implicit, tvd, stream);
    else launch_assemble_of<PREC_FP64>(bp, prev, old, nw, implicit, tvd, stream);
}

void launch_pressure(const BatchPlan &bp, int prec, int prev, int old, int nw, void *stream)
{
    if (prec == PREC_DF64) launch_pressure_of<PREC_DF64>(bp, prev, old, nw, stream);
    else if (prec == PREC_MIXED) launch_pressure_of<PREC_MIXED>(bp, prev, old, nw, stream);
    else launch_pressure_of<PREC_FP64>(bp, prev, old, nw, stream);
}

void launch_velocity(const BatchPlan &bp, int prec, int old, int nw, void *stream)
{
    if (prec == PREC_DF64) launch_velocity_of<PREC_DF64>(bp, old, nw, stream);
    else if (prec == PREC_MIXED) launch_velocity_of<PREC_MIXED>(bp, old, nw, stream);
    else launch_velocity_of<PREC_FP64>(bp, old, nw, stream);
}

}  // namespace stg
