// noalloc.cu -- sim_step_noalloc: the SIMPLE-TS time step for callers that
// cannot allocate device memory (see include/simplets_noalloc.h).
//
// All working memory of the call -- geometry flags, grid factor tables, the
// three state levels in the padded layout, the per-iteration scratch of the
// sweep (face densities, pseudo velocities, d coefficients, explicit terms)
// and the residual words -- is carved out of one file-scope device array.
// The sweep itself runs through the same kernels as sim_step, over a
// one-problem tile list that also lives in the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "problem_rules.h"
#include "simplets.h"
#include "simplets_noalloc.h"
#include "stg_common.cuh"

using namespace stg;

namespace {

constexpr size_t kScratchBytes = (size_t)SIM_NOALLOC_SCRATCH_MB << 20;
constexpr int kMaxRects = 64;
constexpr int kMaxDevices = 64;

// The scratch.  In host code `g_scratch` names a host-side stand-in, not a
// device address: the address kernels need comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_lock;

// The device address of the scratch is looked up once per device and CUDA
// context (cudaGetSymbolAddress, with that device current), and looked up
// again when the caller's current context is another one -- after
// cudaDeviceReset, say, the module is loaded anew and the old address is
// stale.  The context is identified by cuCtxGetId, reached through the
// runtime's driver entry points (no link against the driver library).
struct ScratchSlot {
    unsigned long long ctx_id = 0;
    void *ptr = nullptr;
};
ScratchSlot g_slot[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context; false if there is none
// or the driver cannot say.
bool current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch in the current device's current context.
// The first call on a device (or in a new context) looks it up, which can
// load the library's GPU code; later calls in the same context reuse it.
// When the context cannot be identified the address is looked up every call.
sim_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return SIM_ECUDA;
    std::lock_guard<std::mutex> g(g_lock);
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    ScratchSlot &s = g_slot[dev];
    if (!known || !s.ptr || s.ctx_id != id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)
            return SIM_ECUDA;
        // the lookup makes the device's primary context current if none was
        unsigned long long id2 = 0;
        s.ptr = p;
        s.ctx_id = current_context_id(&id2) ? id2 : 0;
    }
    *out = s.ptr;
    return SIM_OK;
}

enum Kind : uint8_t { NK_FLUID, NK_SOLID, NK_WALL, NK_SYMM, NK_INFLOW, NK_OUTFLOW };

struct Setup {
    int nx, ny, pitch;
    int side_kind[4];
    double side_vel[4], side_T[4], body_T;
    int n_rect;
    const int *rect;              // device copy
    const double *in_u, *in_T, *in_p;   // device copies, ny entries
    double u_in, omega;
    uint8_t *kind, *side;         // extended grid
};

__device__ __forceinline__ int nidx(const Setup &s, int i, int j) { return (j + G) * s.pitch + (i + G); }
__device__ __forceinline__ bool nin(const Setup &s, int i, int j)
{
    return i >= -G && i <= s.nx + G && j >= -G && j <= s.ny + G;
}
__device__ __forceinline__ int nkind(const Setup &s, int i, int j) { return nin(s, i, j) ? s.kind[nidx(s, i, j)] : NK_WALL; }
__device__ __forceinline__ bool nfluid(const Setup &s, int i, int j) { return nkind(s, i, j) == NK_FLUID; }
__device__ __forceinline__ bool nwall(const Setup &s, int i, int j)
{
    const int t = nkind(s, i, j);
    return t == NK_SOLID || t == NK_WALL;
}

// Grid factor tables of one axis (the layout of stg::Axis): cell size,
// inverse, the two interpolation weights of face i, the inverse centre
// distance across face i and the three derivative weights of cell i; ghost
// sizes mirror the boundary cells.
__global__ void k_na_axis(int n, const double *dl, double len, double hrdt, double ct1f, double *out)
{
    const int m = n + 2 * G + 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    auto size_at = [&](int qq) {
        int s = qq - G;
        if (s < 0) s = -s - 1;
        if (s >= n) s = 2 * n - 1 - s;
        return dl ? dl[s] : len / n;
    };
    const double di = size_at(q), dm = q > 0 ? size_at(q - 1) : di;
    const double rd = 1.0 / di, wlo = di / (dm + di), whi = dm / (dm + di);
    out[q] = di;
    out[m + q] = rd;
    out[2 * m + q] = wlo;
    out[3 * m + q] = whi;
    out[4 * m + q] = 1.0 / (0.5 * (dm + di));
    out[8 * m + q] = 0.5 * (dm + di);
    out[9 * m + q] = 2.0 * wlo;
    out[10 * m + q] = 2.0 * whi;
    out[11 * m + q] = 0.5 * di;
    out[12 * m + q] = di * hrdt;
    out[13 * m + q] = (2.0 * ct1f) * di;
    out[14 * m + q] = di * (2.0 * hrdt);
    // derivative weights: the interpolation weights of face q+1 (of face q
    // itself for the last entry, which no cell uses)
    const double dn = q + 1 < m ? size_at(q + 1) : di, dc = q + 1 < m ? di : dm;
    const double wlo_n = dn / (dc + dn), whi_n = dc / (dc + dn);
    const double h = 0.5 * rd;
    out[5 * m + q] = h * wlo;
    out[6 * m + q] = h * (wlo_n - whi);
    out[7 * m + q] = h * whi_n;
}

// Cell kinds of the extended grid: S/N ghost rows own the corners.
__global__ void k_na_kind(Setup s)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - G;
    const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - G;
    if (i > s.nx + G || j > s.ny + G) return;
    const int side = j < 0 ? SIM_S : j >= s.ny ? SIM_N : i < 0 ? SIM_W : i >= s.nx ? SIM_E : -1;
    uint8_t t = NK_FLUID;
    if (side >= 0) {
        const int kd = s.side_kind[side];
        t = kd == SIM_BC_WALL ? NK_WALL : kd == SIM_BC_SYMMETRY ? NK_SYMM : kd == SIM_BC_INFLOW ? NK_INFLOW : NK_OUTFLOW;
    } else {
        for (int r = 0; r < s.n_rect; r++) {
            const int *q = s.rect + 4 * r;
            if (i >= q[0] && i < q[2] && j >= q[1] && j < q[3]) t = NK_SOLID;
        }
    }
    s.kind[nidx(s, i, j)] = t;
    s.side[nidx(s, i, j)] = (uint8_t)(side < 0 ? 0 : side);
}

__device__ __forceinline__ bool na_uact(const Setup &s, int i, int j) { return nfluid(s, i - 1, j) && nfluid(s, i, j); }
__device__ __forceinline__ bool na_vact(const Setup &s, int i, int j) { return nfluid(s, i, j - 1) && nfluid(s, i, j); }

// Geometry flags (stg_common.cuh) of every extended position.
__global__ void k_na_flags(Setup s, uint16_t *flag)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - G;
    const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - G;
    if (i > s.nx + G || j > s.ny + G) return;
    uint32_t b = 0;
    if (nfluid(s, i, j)) b |= F_FLUID;
    if (nwall(s, i, j)) b |= F_WALL;
    if (na_uact(s, i, j)) b |= F_UACT;
    if (nwall(s, i - 1, j) && nwall(s, i, j)) b |= F_UWALL;
    if (na_vact(s, i, j)) b |= F_VACT;
    if (nwall(s, i, j - 1) && nwall(s, i, j)) b |= F_VWALL;
    bool cx = true, cy = true, ux = true, uy = true, vx = true, vy = true;
    for (int q = -2; q <= 1; q++) {
        cx = cx && nfluid(s, i + q, j);
        cy = cy && nfluid(s, i, j + q);
        ux = ux && na_uact(s, i + q, j);
        uy = uy && na_uact(s, i, j + q);
        vx = vx && na_vact(s, i + q, j);
        vy = vy && na_vact(s, i, j + q);
    }
    if (cx) b |= F_TCX;
    if (cy) b |= F_TCY;
    if (ux) b |= F_TUX;
    if (uy) b |= F_TUY;
    if (vx) b |= F_TVX;
    if (vy) b |= F_TVY;
    const int i0 = (i >= 0 ? i : i - 31) / 32 * 32;    // 32-wide row segment holding i
    bool inner = true;
    for (int q = -2; q <= 2 && inner; q++)
        for (int r = i0 - 2; r <= i0 + 33 && inner; r++)
            inner = nfluid(s, r, j + q);
    if (inner) b |= F_INTERIOR;
    flag[nidx(s, i, j)] = (uint16_t)b;
}

// Every node of a level: unknowns from the caller's arrays (logical layout),
// other nodes from the boundary rules (wall state, inflow state, zero normal
// velocity on wall faces; outflow and symmetry copies follow in the ghost pass).
__global__ void k_na_fill(Setup s, const double *u_in, const double *v_in, const double *p_in,
                          const double *T_in, Level L)
{
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - G;
    const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - G;
    if (i > s.nx + G || j > s.ny + G) return;
    const int c = nidx(s, i, j), t = nkind(s, i, j);
    const int row = j < 0 ? 0 : (j >= s.ny ? s.ny - 1 : j);
    double p = 1.0, T = 1.0;
    if (t == NK_FLUID) {
        p = p_in[(size_t)j * s.nx + i];
        T = T_in[(size_t)j * s.nx + i];
    } else if (t == NK_SOLID) {
        T = s.body_T;
    } else if (t == NK_WALL) {
        T = s.side_T[s.side[c]];
    } else if (t == NK_INFLOW) {
        p = s.in_p ? s.in_p[row] : 1.0;
        T = s.in_T ? s.in_T[row] : 1.0;
    }
    L.p[c] = p;
    L.T[c] = T;
    L.rho[c] = p / T;
    L.gam[c] = s.omega == 0.5 ? sqrt(T) : pow(T, s.omega);

    const double uin = s.in_u ? s.in_u[row] : s.u_in;
    const int tl = nkind(s, i - 1, j);
    double u = 0.0;
    if (tl == NK_FLUID && t == NK_FLUID) {
        u = u_in[(size_t)j * (s.nx + 1) + i];
    } else if (tl == NK_FLUID || t == NK_FLUID) {
        u = (tl == NK_INFLOW || t == NK_INFLOW) ? uin : 0.0;
    } else if (nwall(s, i - 1, j) && nwall(s, i, j)) {
        const int sl = s.side[nidx(s, i - 1 < -G ? -G : i - 1, j)], sr = s.side[c];
        if (tl == NK_WALL && (sl == SIM_S || sl == SIM_N)) u = s.side_vel[sl];
        else if (t == NK_WALL && (sr == SIM_S || sr == SIM_N)) u = s.side_vel[sr];
    } else if (tl == NK_INFLOW || t == NK_INFLOW) {
        u = uin;
    }
    L.u[c] = u;

    const int tb = nkind(s, i, j - 1);
    double v = 0.0;
    if (tb == NK_FLUID && t == NK_FLUID) {
        v = v_in[(size_t)j * s.nx + i];
    } else if (tb != NK_FLUID && t != NK_FLUID && nwall(s, i, j - 1) && nwall(s, i, j)) {
        const int sb = s.side[nidx(s, i, j - 1 < -G ? -G : j - 1)], st = s.side[c];
        if (tb == NK_WALL && (sb == SIM_W || sb == SIM_E)) v = s.side_vel[sb];
        else if (t == NK_WALL && (st == SIM_W || st == SIM_E)) v = s.side_vel[st];
    }
    L.v[c] = v;
}

// Bump allocator over the scratch (offsets only; nothing is allocated).
// The problem descriptor of the equation kernels and its tile list (every
// tile belongs to problem 0), written from the launch parameters so that no
// host memory is read when the work runs.
__global__ void k_na_plan(Inst I, Inst *dst, int *tiles, int n_tiles)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) *dst = I;
    if (q < n_tiles) tiles[q] = 0;
}

struct Carver {
    unsigned char *base;
    size_t used = 0;
    bool ok = true;
    template <typename T>
    T *take(size_t count)
    {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = count * sizeof(T);
        if (off + bytes > kScratchBytes) {
            ok = false;
            return nullptr;
        }
        used = off + bytes;
        return reinterpret_cast<T *>(base + off);
    }
};

#define NA_TRY(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return SIM_ECUDA;   \
    } while (0)

}  // namespace

extern "C" sim_status sim_step_noalloc(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc, int n_steps,
                                       int scheme, double *d_u, double *d_v, double *d_p, double *d_T,
                                       void *stream, double res_out[4])
{
    // ---------------------------------------------------- validation (host)
    // the checks sim_create applies, then this entry's own limits
    if (!grid || !gas || !bc || !d_u || !d_v || !d_p || !d_T) return SIM_EINVAL;
    if (n_steps < 0 || (scheme & ~3)) return SIM_EINVAL;
    if (check_description(grid, bc, nullptr, 0) != SIM_OK) return SIM_EINVAL;
    if (bc->n_rect > kMaxRects || bc->tol != 0.0 || bc->precision != SIM_FP64) return SIM_EINVAL;
    const int nx = grid->nx, ny = grid->ny;
    // the coefficients and the time step by the rules sim_create applies
    Coef k{};
    double u_in = 0.0, gm = 0.0;
    if (!gas_coefficients(gas, k, u_in, gm)) return SIM_EINVAL;
    k.dt = time_step(grid, bc, u_in, gm);
    k.hrdt = 0.5 / k.dt;
    k.zeta = bc->zeta_coef;
    k.tau = bc->tau_coef;

    // --------------------------------------------------- carve the scratch
    void *base = nullptr;
    sim_status st = scratch_address(&base);
    if (st != SIM_OK) return st;
    const int pitch = ((nx + 2 * G + 1) + 7) / 8 * 8;
    const size_t nelem = (size_t)pitch * (ny + 2 * G + 1);
    const int mx = nx + 2 * G + 1, my = ny + 2 * G + 1;
    Carver cv{(unsigned char *)base};
    double *pool = cv.take<double>(kPoolArrays * nelem);
    uint16_t *flag = cv.take<uint16_t>(nelem);
    uint8_t *kind = cv.take<uint8_t>(nelem);
    uint8_t *side = cv.take<uint8_t>(nelem);
    double *axx = cv.take<double>(kAxisTables * (size_t)mx);
    double *axy = cv.take<double>(kAxisTables * (size_t)my);
    double *cdx = grid->dx ? cv.take<double>(nx) : nullptr;
    double *cdy = grid->dy ? cv.take<double>(ny) : nullptr;
    double *cin = cv.take<double>(3 * (size_t)ny);
    int *crect = cv.take<int>(4 * kMaxRects);
    unsigned long long *res = cv.take<unsigned long long>(4);
    const int tiles_x = (nx + 1 + 31) / 32, n_tiles = tiles_x * ((ny + 1 + 7) / 8);
    Inst *inst = cv.take<Inst>(1);
    int *tiles = cv.take<int>(n_tiles);
    if (!cv.ok) return SIM_ENOMEM;           // the problem does not fit the static scratch

    cudaStream_t s = (cudaStream_t)stream;
    // inputs the set-up kernels read, copied from the caller's host arrays
    if (cdx) NA_TRY(cudaMemcpyAsync(cdx, grid->dx, nx * sizeof(double), cudaMemcpyHostToDevice, s));
    if (cdy) NA_TRY(cudaMemcpyAsync(cdy, grid->dy, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    if (bc->inflow_u) NA_TRY(cudaMemcpyAsync(cin, bc->inflow_u, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    if (bc->inflow_T) NA_TRY(cudaMemcpyAsync(cin + ny, bc->inflow_T, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    if (bc->inflow_p) NA_TRY(cudaMemcpyAsync(cin + 2 * ny, bc->inflow_p, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    if (bc->n_rect) NA_TRY(cudaMemcpyAsync(crect, bc->rect, 4 * bc->n_rect * sizeof(int), cudaMemcpyHostToDevice, s));
    // the scratch keeps the previous call's contents: clear the work arrays
    NA_TRY(cudaMemsetAsync(pool + 18 * nelem, 0, kWorkArrays * nelem * sizeof(double), s));

    Setup su{};
    su.nx = nx; su.ny = ny; su.pitch = pitch;
    for (int q = 0; q < 4; q++) {
        su.side_kind[q] = bc->side_kind[q];
        su.side_vel[q] = bc->side_vel[q];
        su.side_T[q] = bc->side_T[q];
    }
    su.body_T = bc->body_T;
    su.n_rect = bc->n_rect;
    su.rect = crect;
    su.in_u = bc->inflow_u ? cin : nullptr;
    su.in_T = bc->inflow_T ? cin + ny : nullptr;
    su.in_p = bc->inflow_p ? cin + 2 * ny : nullptr;
    su.u_in = u_in;
    su.omega = k.omega;
    su.kind = kind;
    su.side = side;

    Level lv[3];
    double *q = pool;
    for (int l = 0; l < 3; l++) {
        lv[l].u = q; q += nelem; lv[l].v = q; q += nelem; lv[l].p = q; q += nelem;
        lv[l].T = q; q += nelem; lv[l].rho = q; q += nelem; lv[l].gam = q; q += nelem;
    }
    Work w{};
    w.ru_dy = q; q += nelem; w.rv_dx = q; q += nelem;
    w.Fx = q; q += nelem; w.Fy = q; q += nelem; w.DTx = q; q += nelem; w.DTy = q; q += nelem;
    w.Bgc = q; q += nelem; w.Bgx = q; q += nelem; w.Bgy = q; q += nelem;
    w.Fbu = q; q += nelem; w.Fbv = q; q += nelem;
    w.Su = q; q += nelem; w.Sv = q; q += nelem;
    w.uhat = q; q += nelem; w.du = q; q += nelem;
    w.vhat = q; q += nelem; w.dv = q; q += nelem; w.uexp = q; q += nelem; w.vexp = q; q += nelem;
    w.Texp = q;
    q += nelem;
    double **lim[8] = {&w.psTx, &w.psTy, &w.psUx, &w.psUyU, &w.psUyD, &w.psVy, &w.psVxU, &w.psVxD};
    for (double **x : lim) { *x = q; q += nelem; }
    w.bpx = q; q += nelem; w.bpy = q; q += nelem;
    w.Bgcu = q; q += nelem; w.Bgcv = q; q += nelem;
    w.res = res;

    Geo g{};
    g.nx = nx; g.ny = ny; g.pitch = pitch; g.flag = flag;
    g.x = axis_view<double>(axx, mx);
    g.y = axis_view<double>(axy, my);
    Sides sides{};
    for (int t = 0; t < 4; t++) sides.kind[t] = bc->side_kind[t];

    // -------------------------------------------------------- set-up kernels
    k_na_axis<<<(mx + 127) / 128, 128, 0, s>>>(nx, cdx, grid->lx, k.hrdt, k.CT1f, axx);
    k_na_axis<<<(my + 127) / 128, 128, 0, s>>>(ny, cdy, grid->ly, k.hrdt, k.CT1f, axy);
    const dim3 bl(32, 8), gr((mx + 31) / 32, (my + 7) / 8);
    k_na_kind<<<gr, bl, 0, s>>>(su);
    k_na_flags<<<gr, bl, 0, s>>>(su, flag);
    k_na_fill<<<gr, bl, 0, s>>>(su, d_u, d_v, d_p, d_T, lv[0]);
    launch_derive(g, k, lv[0], s);
    launch_ghosts(g, sides, lv[0], false, s);
    for (int l = 1; l < 3; l++)
        for (int f = 0; f < 6; f++) {
            double *dst = f == 0 ? lv[l].u : f == 1 ? lv[l].v : f == 2 ? lv[l].p : f == 3 ? lv[l].T : f == 4 ? lv[l].rho : lv[l].gam;
            const double *src = f == 0 ? lv[0].u : f == 1 ? lv[0].v : f == 2 ? lv[0].p : f == 3 ? lv[0].T : f == 4 ? lv[0].rho : lv[0].gam;
            NA_TRY(cudaMemcpyAsync(dst, src, nelem * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
    NA_TRY(cudaMemsetAsync(res, 0, 4 * sizeof(unsigned long long), s));

    Inst one{};
    one.g = g;
    one.k = k;
    for (int l = 0; l < 3; l++) one.lv[l] = lv[l];
    one.w = w;
    one.east_outflow = bc->side_kind[SIM_E] == SIM_BC_OUTFLOW;
    one.tiles_x = tiles_x;
    one.tile0 = 0;
    k_na_plan<<<(n_tiles + 255) / 256, 256, 0, s>>>(one, inst, tiles, n_tiles);
    const BatchPlan plan{inst, tiles, 1, n_tiles, 32, 8, n_tiles, one, 0};

    // ------------------------------------------------- the time steps (S0-S9)
    const bool implicit = scheme & SIM_IMPLICIT, tvd = scheme & SIM_TVD;
    int cur = 0;
    for (int step = 0; step < n_steps; step++) {
        const int prev = cur;
        int old = prev;
        if (!implicit) {
            launch_faces(plan, PREC_FP64, prev, tvd, true, s);
            launch_explicit(plan, PREC_FP64, prev, tvd, s);
        }
        for (int it = 0; it < bc->iters; it++) {
            int nw = (old + 1) % 3;
            if (nw == prev) nw = (nw + 1) % 3;
            if (implicit || it > 0)     // an explicit step's first iteration reuses the faces of n-1
                launch_faces(plan, PREC_FP64, old, tvd, implicit, s);
            launch_assemble(plan, PREC_FP64, prev, old, nw, implicit, tvd, s);
            launch_pressure(plan, PREC_FP64, prev, old, nw, s);
            launch_velocity(plan, PREC_FP64, old, nw, s);
            launch_ghosts(g, sides, lv[nw], true, s);
            old = nw;
        }
        cur = old;
    }
    launch_gather(g, SIM_FIELD_U, lv[cur], d_u, s);
    launch_gather(g, SIM_FIELD_V, lv[cur], d_v, s);
    launch_gather(g, SIM_FIELD_P, lv[cur], d_p, s);
    launch_gather(g, SIM_FIELD_T, lv[cur], d_T, s);
    NA_TRY(cudaGetLastError());
    if (res_out) {
        unsigned long long h[4];
        NA_TRY(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, s));
        NA_TRY(cudaStreamSynchronize(s));
        bool bad = false;
        for (int t = 0; t < 4; t++) {
            std::memcpy(&res_out[t], &h[t], sizeof(double));
            if (!std::isfinite(res_out[t])) bad = true;
        }
        if (bad) return SIM_EDIVERGED;
    }
    return SIM_OK;
}
