// simplets_host.cu -- host side of the C ABI declared in include/simplets.h:
// problem validation, the non-dimensional coefficients, geometry flags, the
// start state, device memory and the loop-1 / loop-2 driver of SIMPLE-TS
// (arXiv:1802.04243, Section 3.1).  Every arithmetic step of the sweep runs in
// the kernels of phase_kernels.cuh and sweep_kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "problem_rules.h"
#include "simplets.h"
#include "stg_common.cuh"

using namespace stg;

namespace {

enum CellKind { K_FLUID, K_SOLID, K_WALL, K_SYMM, K_INFLOW, K_OUTFLOW };

struct Problem {
    int nx, ny;
    std::vector<double> dx, dy;                // logical cell sizes
    int side_kind[4];
    double side_vel[4], side_T[4], body_T;
    std::vector<int> rect;                     // 4 per obstacle
    std::vector<double> in_u, in_T, in_p;      // per row
    double u_in, gamma;
    Coef k;
    int iters;
    double tol;
    uint64_t seed;
    double perturb;
    int precision;
};

}  // namespace

struct sim_s {
    Problem pb;
    int pitch = 0;
    size_t nelem = 0;                          // elements of one extended field
    // x-window of the handle: it stores the columns [win_L, win_R) of the
    // extended grid (a whole problem: [-2, nx + 3)) and computes the positions
    // of the columns [win_L + 2, win_R - 2); a strip of an x-decomposed
    // problem (sim_strips_create) stores a window.  The device arrays the
    // kernels see are the allocations moved back by `shift` elements, so that
    // element (i, j) keeps its whole-problem index (j + 2) pitch + (i + 2).
    int win_L = -G, win_R = 0;
    long shift = 0;
    int own0 = 0, own_stop = 0;                // columns whose residuals count (own_stop 0: no limit)
    cudaStream_t stream = nullptr;
    Geo geo{};
    Sides sides{};
    Level lv[3]{};
    Work work{};
    double *d_pool = nullptr;                  // every double array of the handle
    uint16_t *d_flag = nullptr;
    double *d_axis = nullptr;
    double *d_stage = nullptr;                 // logical-shape staging array
    double *d_state = nullptr;                 // u, v, p, T staged back to back (allocated on first use)
    unsigned *d_bad = nullptr;                 // admissibility flag of a staged state
    unsigned *h_bad = nullptr;                 // its pinned host copy
    // mixed precision: FP32 levels, FP32 scratch and grid factors
    bool mixed = false;
    Mixed mx{};
    bool mx_dirty = false;                     // the FP64 u, v, T, Gamma lag behind the FP32 ones (mixed)
    float *d_pool32 = nullptr;
    float *d_axis32 = nullptr;
    // double-float precision: working levels, scratch and grid factors; the
    // FP64 levels are refreshed from them when the state is read out
    bool df = false;
    bool df_dirty = false;                     // the FP64 levels lag behind the double-float ones
    DoubleFloat dfm{};
    df64 *d_pooldf = nullptr;
    df64 *d_axisdf = nullptr;
    // the one-problem tile list the equation kernels walk (32 x 8 tiles)
    Inst *d_inst = nullptr;
    int *d_tiles = nullptr;
    BatchPlan plan{};
    unsigned long long *h_res = nullptr;       // pinned copy of the residuals
    int cur = 0;                               // level holding the current state
    int last_iters = 0;
    bool diverged = false;
    unsigned set_mask = 0;
    // measurement hooks
    long long launches[SIM_K_COUNT] = {0};
    bool timing = false;
    struct Mark { int cls; cudaEvent_t e0, e1; };
    std::vector<Mark> marks;                   // recorded launches (timing on)
    std::vector<cudaEvent_t> spare;            // reusable events
    // CUDA graphs of one time step, per (start level, scheme)
    struct StepGraph { cudaGraphExec_t exec = nullptr; int result = 0; long long counts[SIM_K_COUNT] = {0}; };
    StepGraph graphs[3][4];
    cudaStream_t cap_stream = nullptr;         // private stream the step graphs are captured on
    bool graphs_off = false;
    char err[256] = {0};
};

namespace {

sim_status fail(sim_t s, sim_status st, const char *fmt, ...)
{
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->err, sizeof s->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define CUDA_TRY(sim, call)                                                          \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(sim, SIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// splitmix64 (Steele, Lea and Flood, 2014) used as a counter hash of
// (seed, field, i, j); returns a double in [-1, 1).
double hash_uniform(uint64_t seed, int field, int i, int j)
{
    uint64_t z = seed ^ (((uint64_t)field << 40) + ((uint64_t)j << 20) + (uint64_t)i);
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

// Non-dimensional parameters (Section 4 scaling; Eq. pl37 for the hard-sphere
// gas), by the rules of problem_rules.h.
sim_status derive_coefficients(const sim_gas *gas, Problem &pb, sim_t err)
{
    if (!gas_coefficients(gas, pb.k, pb.u_in, pb.gamma)) {
        if (gas->model == SIM_GAS_IDEAL_RE)
            return fail(err, SIM_EINVAL, "ideal gas needs reynolds > 0, gamma > 1, prandtl > 0");
        return fail(err, SIM_EINVAL, "unknown gas model %d", gas->model);
    }
    return SIM_OK;
}

sim_status read_problem(const sim_grid *gr, const sim_gas *gas, const sim_bc *bc, Problem &pb, sim_t err)
{
    if (!gas) return fail(err, SIM_EINVAL, "null description");
    char msg[200];
    if (check_description(gr, bc, msg, sizeof msg) != SIM_OK) return fail(err, SIM_EINVAL, "%s", msg);
    pb.nx = gr->nx;
    pb.ny = gr->ny;
    pb.dx.resize(pb.nx);
    pb.dy.resize(pb.ny);
    for (int i = 0; i < pb.nx; i++) pb.dx[i] = gr->dx ? gr->dx[i] : gr->lx / pb.nx;
    for (int j = 0; j < pb.ny; j++) pb.dy[j] = gr->dy ? gr->dy[j] : gr->ly / pb.ny;
    for (int s = 0; s < 4; s++) {
        pb.side_kind[s] = bc->side_kind[s];
        pb.side_vel[s] = bc->side_vel[s];
        pb.side_T[s] = bc->side_T[s];
    }
    pb.body_T = bc->body_T;
    for (int r = 0; r < bc->n_rect; r++) pb.rect.insert(pb.rect.end(), bc->rect + 4 * r, bc->rect + 4 * r + 4);
    pb.iters = bc->iters;
    pb.tol = bc->tol;
    pb.seed = bc->seed;
    pb.perturb = bc->perturb;
    pb.precision = bc->precision;
    sim_status st = derive_coefficients(gas, pb, err);
    if (st != SIM_OK) return st;
    pb.k.zeta = bc->zeta_coef;
    pb.k.tau = bc->tau_coef;
    pb.in_u.resize(pb.ny);
    pb.in_T.resize(pb.ny);
    pb.in_p.resize(pb.ny);
    for (int j = 0; j < pb.ny; j++) {
        pb.in_u[j] = bc->inflow_u ? bc->inflow_u[j] : pb.u_in;
        pb.in_T[j] = bc->inflow_T ? bc->inflow_T[j] : 1.0;
        pb.in_p[j] = bc->inflow_p ? bc->inflow_p[j] : 1.0;
    }
    // time step: given, or cfl * min cell size / (U_ref + sound speed)
    pb.k.dt = time_step(gr, bc, pb.u_in, pb.gamma);
    pb.k.hrdt = 0.5 / pb.k.dt;
    return SIM_OK;
}

// ----------------------------------------------------------- host geometry

struct HostGrid {
    int nx, ny, P;
    std::vector<uint8_t> kind, side;           // over [-2, nx+2] x [-2, ny+2]
    int at(int i, int j) const { return (j + G) * P + (i + G); }
    bool in(int i, int j) const { return i >= -G && i <= nx + G && j >= -G && j <= ny + G; }
    int k(int i, int j) const { return in(i, j) ? (int)kind[at(i, j)] : (int)K_WALL; }
    // side of the nearest position of the extended grid (lookups one layer
    // beyond it, from the faces of the outermost ghost layer, stay inside)
    int side_at(int i, int j) const
    {
        i = i < -G ? -G : (i > nx + G ? nx + G : i);
        j = j < -G ? -G : (j > ny + G ? ny + G : j);
        return side[at(i, j)];
    }
    bool fluid(int i, int j) const { return k(i, j) == K_FLUID; }
    bool wall(int i, int j) const { int t = k(i, j); return t == K_SOLID || t == K_WALL; }
};

void classify(const Problem &pb, HostGrid &h)
{
    h.kind.assign((size_t)h.P * (pb.ny + 2 * G + 1), K_WALL);
    h.side.assign(h.kind.size(), 0);
    for (int j = -G; j <= pb.ny + G; j++)
        for (int i = -G; i <= pb.nx + G; i++) {
            int side = j < 0 ? SIM_S : j >= pb.ny ? SIM_N : i < 0 ? SIM_W : i >= pb.nx ? SIM_E : -1;
            uint8_t t = K_FLUID;
            if (side >= 0) {
                switch (pb.side_kind[side]) {
                case SIM_BC_WALL: t = K_WALL; break;
                case SIM_BC_SYMMETRY: t = K_SYMM; break;
                case SIM_BC_INFLOW: t = K_INFLOW; break;
                default: t = K_OUTFLOW; break;
                }
            }
            h.kind[h.at(i, j)] = t;
            h.side[h.at(i, j)] = (uint8_t)(side < 0 ? 0 : side);
        }
    for (size_t r = 0; r < pb.rect.size(); r += 4)
        for (int j = pb.rect[r + 1]; j < pb.rect[r + 3]; j++)
            for (int i = pb.rect[r]; i < pb.rect[r + 2]; i++)
                h.kind[h.at(i, j)] = K_SOLID;
}

std::vector<uint16_t> make_flags(const HostGrid &h)
{
    std::vector<uint16_t> f(h.kind.size(), 0);
    auto uact = [&](int i, int j) { return h.fluid(i - 1, j) && h.fluid(i, j); };
    auto vact = [&](int i, int j) { return h.fluid(i, j - 1) && h.fluid(i, j); };
    for (int j = -G; j <= h.ny + G; j++)
        for (int i = -G; i <= h.nx + G; i++) {
            uint32_t b = 0;
            if (h.fluid(i, j)) b |= F_FLUID;
            if (h.wall(i, j)) b |= F_WALL;
            if (uact(i, j)) b |= F_UACT;
            if (h.wall(i - 1, j) && h.wall(i, j)) b |= F_UWALL;
            if (vact(i, j)) b |= F_VACT;
            if (h.wall(i, j - 1) && h.wall(i, j)) b |= F_VWALL;
            bool cx = true, cy = true, ux = true, uy = true, vx = true, vy = true;
            for (int q = -2; q <= 1; q++) {
                cx = cx && h.fluid(i + q, j);
                cy = cy && h.fluid(i, j + q);
                ux = ux && uact(i + q, j);
                uy = uy && uact(i, j + q);
                vx = vx && vact(i + q, j);
                vy = vy && vact(i, j + q);
            }
            if (cx) b |= F_TCX;
            if (cy) b |= F_TCY;
            if (ux) b |= F_TUX;
            if (uy) b |= F_TUY;
            if (vx) b |= F_TVX;
            if (vy) b |= F_TVY;
            // the 32-wide row segment holding i has no wall within two cells
            const int i0 = (i >= 0 ? i : i - 31) / 32 * 32;
            bool inner = true;
            for (int q = -2; q <= 2 && inner; q++)
                for (int r = i0 - 2; r <= i0 + 33 && inner; r++)
                    inner = h.fluid(r, j + q);
            if (inner) b |= F_INTERIOR;
            f[h.at(i, j)] = (uint16_t)b;
        }
    return f;
}

// Axis factor table: kAxisTables arrays of n + 2G + 1 entries over [-2, n+2];
// hrdt = 1 / (2 dt), ct1f = C^T1_f.
std::vector<double> make_axis(const std::vector<double> &dl, double hrdt, double ct1f)
{
    const int n = (int)dl.size(), m = n + 2 * G + 1;
    std::vector<double> d(m), out(kAxisTables * (size_t)m, 0.0);
    for (int i = -G; i <= n + G; i++) {
        int s = i;
        if (s < 0) s = -s - 1;                  // mirror about the west / south side
        if (s >= n) s = 2 * n - 1 - s;          // mirror about the east / north side
        d[i + G] = dl[s];
    }
    for (int q = 0; q < m; q++) {
        const double di = d[q], dm = q > 0 ? d[q - 1] : d[q];
        out[q] = di;
        out[m + q] = 1.0 / di;
        out[2 * m + q] = di / (dm + di);
        out[3 * m + q] = dm / (dm + di);
        out[4 * m + q] = 1.0 / (0.5 * (dm + di));
        out[8 * m + q] = 0.5 * (dm + di);
        out[9 * m + q] = 2.0 * out[2 * m + q];
        out[10 * m + q] = 2.0 * out[3 * m + q];
        out[11 * m + q] = 0.5 * di;
        out[12 * m + q] = di * hrdt;
        out[13 * m + q] = (2.0 * ct1f) * di;
        out[14 * m + q] = di * (2.0 * hrdt);      // 2 hrdt = 1 / dt exactly
    }
    for (int q = 0; q < m; q++) {
        const int qn = q + 1 < m ? q + 1 : q;
        const double h = 0.5 * out[m + q];
        out[5 * m + q] = h * out[2 * m + q];
        out[6 * m + q] = h * (out[2 * m + qn] - out[3 * m + q]);
        out[7 * m + q] = h * out[3 * m + qn];
    }
    return out;
}

double gamma_of(const Problem &pb, double T) { return pb.k.omega == 0.5 ? std::sqrt(T) : std::pow(T, pb.k.omega); }

// Stored values of every node that is not an unknown, and the start state of
// the unknowns (inflow state of the row plus the seeded perturbation).
void build_start_level(const Problem &pb, const HostGrid &h, std::vector<double> *f /* u v p T rho gam */)
{
    const int nx = pb.nx, ny = pb.ny;
    const bool inflow = pb.side_kind[SIM_W] == SIM_BC_INFLOW;
    auto row = [&](int j) { return j < 0 ? 0 : (j >= ny ? ny - 1 : j); };
    for (int j = -G; j <= ny + G; j++)
        for (int i = -G; i <= nx + G; i++) {
            const int c = h.at(i, j);
            const int t = h.k(i, j);
            double p = 1.0, T = 1.0;
            if (t == K_FLUID) {
                if (inflow) { p = pb.in_p[j]; T = pb.in_T[j]; }
                p *= 1.0 + pb.perturb * hash_uniform(pb.seed, 2, i, j);
                T *= 1.0 + pb.perturb * hash_uniform(pb.seed, 3, i, j);
            } else if (t == K_SOLID) {
                T = pb.body_T;
            } else if (t == K_WALL) {
                T = pb.side_T[h.side[c]];
            } else if (t == K_INFLOW) {
                p = pb.in_p[row(j)];
                T = pb.in_T[row(j)];
            }
            f[2][c] = p;
            f[3][c] = T;
            f[4][c] = p / T;
            f[5][c] = gamma_of(pb, T);

            // u face between cells (i-1, j) and (i, j)
            const int tl = h.k(i - 1, j), tr = t;
            double u = 0.0;
            if (tl == K_FLUID && tr == K_FLUID) {
                u = (inflow ? pb.in_u[j] : 0.0) * (1.0 + pb.perturb * hash_uniform(pb.seed, 0, i, j));
            } else if (tl == K_FLUID || tr == K_FLUID) {
                u = (tl == K_INFLOW || tr == K_INFLOW) ? pb.in_u[row(j)] : 0.0;
            } else if (h.wall(i - 1, j) && h.wall(i, j)) {
                // inside a wall: tangential wall speed behind a S/N wall, else 0
                int sl = h.side_at(i - 1, j), sr = h.side[c];
                if (tl == K_WALL && (sl == SIM_S || sl == SIM_N)) u = pb.side_vel[sl];
                else if (tr == K_WALL && (sr == SIM_S || sr == SIM_N)) u = pb.side_vel[sr];
            } else if (tl == K_INFLOW || tr == K_INFLOW) {
                u = pb.in_u[row(j)];
            }
            f[0][c] = u;

            // v face between cells (i, j-1) and (i, j)
            const int tb = h.k(i, j - 1), tt = t;
            double v = 0.0;
            if (tb == K_FLUID && tt == K_FLUID) {
                v = pb.perturb * pb.u_in * hash_uniform(pb.seed, 1, i, j);
            } else if (tb != K_FLUID && tt != K_FLUID && h.wall(i, j - 1) && h.wall(i, j)) {
                int sb = h.side_at(i, j - 1), st = h.side[c];
                if (tb == K_WALL && (sb == SIM_W || sb == SIM_E)) v = pb.side_vel[sb];
                else if (tt == K_WALL && (st == SIM_W || st == SIM_E)) v = pb.side_vel[st];
            }
            f[1][c] = v;
        }
}

double *level_field(const Level &L, int f)
{
    switch (f) {
    case SIM_FIELD_U: return L.u;
    case SIM_FIELD_V: return L.v;
    case SIM_FIELD_P: return L.p;
    case SIM_FIELD_T: return L.T;
    case SIM_FIELD_RHO: return L.rho;
    default: return L.gam;
    }
}

// The problem as the equation kernels see it, cut into tiles of tx x ty
// threads that start at entry `tile0` of the tile list.
Inst inst_of(const sim_s *s, int tx, int tile0)
{
    Inst I{};
    I.g = s->geo;
    I.k = s->pb.k;
    I.g32 = s->mx.g;
    I.k32 = s->mx.k;
    for (int l = 0; l < 3; l++) {
        I.lv[l] = s->lv[l];
        I.lv32[l] = s->mx.lv[l];
    }
    I.w = s->work;
    I.w32 = s->mx.w;
    I.gdf = s->dfm.g;
    I.kdf = s->dfm.k;
    for (int l = 0; l < 3; l++) I.lvdf[l] = s->dfm.lv[l];
    I.wdf = s->dfm.w;
    I.east_outflow = s->sides.kind[SIDE_E] == BC_OUTFLOW;
    const int c0 = s->win_L + G, c1 = s->win_R - G;
    I.tiles_x = (c1 - c0 + tx - 1) / tx;
    I.tile0 = tile0;
    I.x0 = c0;
    I.x_stop = c1 < s->pb.nx + 1 ? c1 : 0;
    I.own0 = s->own0;
    I.own_stop = s->own_stop;
    return I;
}

int prec_of(const sim_s *s) { return s->mixed ? PREC_MIXED : s->df ? PREC_DF64 : PREC_FP64; }

// A pool holds three levels of six fields, then the iteration scratch
// (WorkT, kWorkArrays arrays), which starts at ru_dy and is cleared at
// creation.

// Carve three state levels and the iteration scratch out of one pool.
template <typename R>
R *carve_levels(R *q, size_t nelem, LevelT<R> lv[3], WorkT<R> &w)
{
    for (int l = 0; l < 3; l++) {
        R **f[6] = {&lv[l].u, &lv[l].v, &lv[l].p, &lv[l].T, &lv[l].rho, &lv[l].gam};
        for (R **x : f) { *x = q; q += nelem; }
    }
    R **a[kWorkArrays] = {&w.ru_dy, &w.rv_dx, &w.Fx, &w.Fy, &w.DTx, &w.DTy, &w.Bgc, &w.Bgx, &w.Bgy,
                          &w.Fbu, &w.Fbv, &w.Su, &w.Sv, &w.uhat, &w.du, &w.vhat, &w.dv, &w.uexp, &w.vexp, &w.Texp,
                          &w.psTx, &w.psTy, &w.psUx, &w.psUyU, &w.psUyD, &w.psVy, &w.psVxU, &w.psVxD,
                          &w.bpx, &w.bpy, &w.Bgcu, &w.Bgcv};
    for (R **x : a) { *x = q; q += nelem; }
    return q;
}

// The arrays of a level and of the iteration scratch as kernel views: each
// pointer moved back by d elements (see sim_s::shift); d = 0 for a whole
// problem.
template <typename R>
void shift_views(LevelT<R> lv[3], WorkT<R> &w, long d)
{
    for (int l = 0; l < 3; l++) {
        R **f[6] = {&lv[l].u, &lv[l].v, &lv[l].p, &lv[l].T, &lv[l].rho, &lv[l].gam};
        for (R **x : f) *x -= d;
    }
    R **a[kWorkArrays] = {&w.ru_dy, &w.rv_dx, &w.Fx, &w.Fy, &w.DTx, &w.DTy, &w.Bgc, &w.Bgx, &w.Bgy,
                          &w.Fbu, &w.Fbv, &w.Su, &w.Sv, &w.uhat, &w.du, &w.vhat, &w.dv, &w.uexp, &w.vexp, &w.Texp,
                          &w.psTx, &w.psTy, &w.psUx, &w.psUyU, &w.psUyD, &w.psVy, &w.psVxU, &w.psVxD,
                          &w.bpx, &w.bpy, &w.Bgcu, &w.Bgcv};
    for (R **x : a) *x -= d;
}

// A kernel view of a level back to its allocation (whole-array operations).
template <typename R>
LevelT<R> alloc_of(const LevelT<R> &v, long d)
{
    return LevelT<R>{v.u + d, v.v + d, v.p + d, v.T + d, v.rho + d, v.gam + d};
}

// The FP64 level of the current state brought up to date: from the
// double-float level, or in the mixed path the FP64 u, v, T and Gamma, which
// its sweep keeps in FP32 only (then the ghost refresh that follows a
// velocity update, so the FP64 ghosts match too).
void sync_out(sim_t s)
{
    if (s->df && s->df_dirty) {
        launch_join(s->dfm.lv[s->cur], s->lv[s->cur], s->nelem, s->stream);
        s->df_dirty = false;
    }
    if (s->mixed && s->mx_dirty) {
        launch_widen_mixed(s->geo, s->lv[s->cur], s->mx.lv[s->cur], s->sides.kind[SIDE_E] == BC_OUTFLOW, 0,
                           s->pb.nx + 1, s->stream);
        launch_ghosts(s->geo, s->sides, s->lv[s->cur], true, s->stream);
        s->mx_dirty = false;
    }
}

// Tiles of tx x ty positions over the positions a handle computes: the
// (nx + 1) x (ny + 1) positions of a problem, the columns of a strip's window.
int tiles_of(const sim_s *s, int tx, int ty)
{
    const int w = s->win_R - s->win_L - 2 * G;
    return ((w + tx - 1) / tx) * ((s->pb.ny + 1 + ty - 1) / ty);
}

// Tile shapes the tile-list kernels accept: tx in {16, 32, 64, 128, 256},
// tx * ty in {32, 64, 128, 256} threads.
bool plan_shape_ok(int tx, int ty, int ctas)
{
    const int threads = tx * ty;
    return (tx == 16 || tx == 32 || tx == 64 || tx == 128 || tx == 256) && ty >= 1 &&
           (threads == 32 || threads == 64 || threads == 128 || threads == 256) && ctas >= 0;
}

void drop_step_graphs(sim_t s)
{
    for (auto &row : s->graphs)
        for (auto &g : row)
            if (g.exec) {
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
            }
}

// The one-problem tile list of a handle: tiles of tx x ty threads, `ctas`
// CTAs walking the list (0: one per tile), the assembly kernel `asm_ctas`
// (0: as the others).  The step graphs, which hold the old list, are rebuilt
// on the next step.
sim_status single_plan(sim_t s, int tx, int ty, int ctas, int asm_ctas)
{
    const Inst one = inst_of(s, tx, 0);
    const int ntiles = tiles_of(s, tx, ty);
    CUDA_TRY(s, cudaMemcpyAsync(s->d_inst, &one, sizeof(Inst), cudaMemcpyHostToDevice, s->stream));
    s->plan = BatchPlan{s->d_inst, s->d_tiles, 1, ntiles, tx, ty, ctas > 0 ? std::min(ctas, ntiles) : ntiles, one,
                        asm_ctas > 0 ? std::min(asm_ctas, ntiles) : 0};
    drop_step_graphs(s);
    return SIM_OK;
}

// The measured best distribution per arithmetic on the 4864x1216 channel
// (bench.py --sweep plans):
// - FP64: tiles of 32 x 4 threads, one CTA per tile;
// - mixed: tiles of 32 x 8, one CTA per tile, and for the FP32 assembly as
//   many CTAs as stay resident (1024 threads per SM at its 64 registers)
//   walking the tiles (6375 Mcell-steps/s against 6165 with 32 x 4 tiles:
//   the velocity kernel, 0.101 -> 0.082 ms, ends half as many CTAs, each
//   with its residual atomics);
// - double-float: 32 x 8, one CTA per tile.
sim_status default_plan(sim_t s)
{
    const int prec = prec_of(s);
    if (prec == PREC_DF64) return single_plan(s, 32, 8, 0, 0);
    if (prec == PREC_FP64) return single_plan(s, 32, 4, 0, 0);
    const int tx = 32, ty = 8;
    int dev = 0, sms = 0, asm_ctas = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        asm_ctas = 1024 / (tx * ty) * sms;
    return single_plan(s, tx, ty, 0, asm_ctas);
}

size_t field_count(const Problem &pb, int f)
{
    const size_t nx = pb.nx, ny = pb.ny;
    return f == SIM_FIELD_U ? (nx + 1) * ny : f == SIM_FIELD_V ? nx * (ny + 1) : nx * ny;
}

cudaEvent_t take_event(sim_t s)
{
    if (!s->spare.empty()) {
        cudaEvent_t e = s->spare.back();
        s->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one kernel launch of the direct path: counts it, and times it when
// timing is on.  Under stream capture (counts != nullptr) it only counts.
struct Launch {
    sim_t s;
    int cls;
    cudaStream_t st;
    long long *counts;
    cudaEvent_t e0 = nullptr;
    Launch(sim_t s_, int c, cudaStream_t st_, long long *counts_, int n = 1) : s(s_), cls(c), st(st_), counts(counts_)
    {
        (counts ? counts : s->launches)[cls] += n;
        if (s->timing && !counts) {
            e0 = take_event(s);
            cudaEventRecord(e0, st);
        }
    }
    ~Launch()
    {
        if (e0) {
            cudaEvent_t e1 = take_event(s);
            cudaEventRecord(e1, st);
            s->marks.push_back({cls, e0, e1});
        }
    }
};

// Explicit convective terms of the step that starts from level `prev`
// (explicit scheme only, once per step).  counts != nullptr: capture mode.
void enqueue_explicit(sim_t s, int prev, bool tvd, cudaStream_t st, long long *counts)
{
    { Launch l(s, SIM_K_FACES, st, counts); launch_faces(s->plan, prec_of(s), prev, tvd, true, st); }
    { Launch l(s, SIM_K_EXPLICIT, st, counts); launch_explicit(s->plan, prec_of(s), prev, tvd, st); }
}

// One loop-2 iteration from level `old` (level `prev` holds n-1) into the
// third level, which is returned.  faces_ready: the face quantities of `old`
// are already in the scratch (the first iteration of an explicit step, whose
// explicit terms were computed from the same level), so the face kernel is
// not launched again.
int enqueue_iteration(sim_t s, int prev, int old, bool implicit, bool tvd, bool faces_ready, cudaStream_t st,
                      long long *counts)
{
    int nw = (old + 1) % 3;
    if (nw == prev) nw = (nw + 1) % 3;
    const int ng = ghost_kernels(s->sides, true);
    const int prec = prec_of(s);
    if (!faces_ready) { Launch l(s, SIM_K_FACES, st, counts); launch_faces(s->plan, prec, old, tvd, implicit, st); }
    { Launch l(s, SIM_K_ASSEMBLE, st, counts); launch_assemble(s->plan, prec, prev, old, nw, implicit, tvd, st); }
    { Launch l(s, SIM_K_PRESSURE, st, counts); launch_pressure(s->plan, prec, prev, old, nw, st); }
    { Launch l(s, SIM_K_VELOCITY, st, counts); launch_velocity(s->plan, prec, old, nw, st); }
    if (ng) {
        Launch l(s, SIM_K_GHOSTS, st, counts, s->mixed ? 2 * ng : ng);
        if (s->df) {
            launch_ghosts_df(s->dfm, s->sides, nw, true, st);
        } else {
            launch_ghosts(s->geo, s->sides, s->lv[nw], true, st);
            if (s->mixed) launch_ghosts_f32(s->mx, s->sides, nw, true, st);
        }
    }
    return nw;
}

// One time step from level `prev` with `iters` loop-2 iterations; returns the
// level holding the result.
int enqueue_step(sim_t s, int prev, bool implicit, bool tvd, cudaStream_t st, long long *counts)
{
    if (!implicit) enqueue_explicit(s, prev, tvd, st, counts);
    int old = prev;
    for (int it = 1; it <= s->pb.iters; it++)
        old = enqueue_iteration(s, prev, old, implicit, tvd, !implicit && it == 1, st, counts);
    return old;
}

sim_status check_live(sim_t s)
{
    if (!s) return SIM_EINVAL;
    if (s->diverged) return fail(s, SIM_ESTATE, "handle is in the error state after a divergence");
    return SIM_OK;
}

}  // namespace

// ====================================================================== ABI

namespace {

// Host-side set-up of a whole problem, shared by every handle built from it
// (one for sim_create, one per strip for sim_strips_create): the geometry
// flags, the axis tables and the start state over the extended grid with the
// whole problem's row pitch gP.
struct Template {
    int gP = 0;
    HostGrid h;
    std::vector<uint16_t> flags;
    std::vector<double> ax, ay;
    std::vector<double> f[6];                  // u v p T rho gam
};

void make_template(const Problem &pb, Template &t)
{
    t.gP = ((pb.nx + 2 * G + 1) + 7) / 8 * 8;
    t.h.nx = pb.nx;
    t.h.ny = pb.ny;
    t.h.P = t.gP;
    classify(pb, t.h);
    t.flags = make_flags(t.h);
    t.ax = make_axis(pb.dx, pb.k.hrdt, pb.k.CT1f);
    t.ay = make_axis(pb.dy, pb.k.hrdt, pb.k.CT1f);
    const size_t n = (size_t)t.gP * (pb.ny + 2 * G + 1);
    for (auto &a : t.f) a.assign(n, 0.0);
    build_start_level(pb, t.h, t.f);
}

// Allocate and fill the device side of a handle whose problem (s->pb) and
// stream are set: the columns [L, R) of the extended grid (a whole problem:
// L = -2, R = nx + 3), with the window's slices of the template's flags and
// start state, the whole axis tables, rho and Gamma derived on the device,
// ghosts refreshed, shadow levels of the mixed and double-float paths.  On
// failure the caller destroys s.
sim_status build_handle(sim_t s, const Template &t, int L, int R)
{
    const Problem &pb = s->pb;
    s->win_L = L;
    s->win_R = R;
    s->shift = L + G;
    s->pitch = ((R - L) + 7) / 8 * 8;
    const int rows = pb.ny + 2 * G + 1;
    s->nelem = (size_t)s->pitch * rows;
    const bool whole = L == -G && R == pb.nx + G + 1;

    // the window's slices (the whole arrays for a whole problem)
    std::vector<uint16_t> wflags;
    std::vector<double> wf[6];
    const std::vector<uint16_t> *flags = &t.flags;
    const std::vector<double> *f = t.f;
    if (!whole) {
        wflags.assign(s->nelem, 0);
        for (auto &a : wf) a.assign(s->nelem, 0.0);
        for (int r = 0; r < rows; r++)
            for (int i = L; i < R; i++) {
                const size_t gq = (size_t)r * t.gP + (i + G), lq = (size_t)r * s->pitch + (i - L);
                wflags[lq] = t.flags[gq];
                for (int k = 0; k < 6; k++) wf[k][lq] = t.f[k][gq];
            }
        flags = &wflags;
        f = wf;
    }

    // one pool for 3 levels x 6 fields + the work arrays
    cudaError_t e = cudaMalloc(&s->d_pool, kPoolArrays * s->nelem * sizeof(double));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA;
    Work &w = s->work;
    carve_levels(s->d_pool, s->nelem, s->lv, static_cast<WorkT<double> &>(w));
    const size_t nax = t.ax.size(), nay = t.ay.size();
    const size_t stage = (size_t)(pb.nx + 1) * (pb.ny + 1);
    if (cudaMalloc(&s->d_flag, s->nelem * sizeof(uint16_t)) != cudaSuccess ||
        cudaMalloc(&s->d_axis, (nax + nay) * sizeof(double)) != cudaSuccess ||
        (whole && cudaMalloc(&s->d_stage, stage * sizeof(double)) != cudaSuccess) ||
        cudaMalloc(&w.res, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&s->h_res, 4 * sizeof(unsigned long long)) != cudaSuccess)
        return SIM_ENOMEM;

    s->geo.nx = pb.nx;
    s->geo.ny = pb.ny;
    s->geo.pitch = s->pitch;
    s->geo.flag = s->d_flag - s->shift;
    const int mx = pb.nx + 2 * G + 1, my = pb.ny + 2 * G + 1;
    const double *dax = s->d_axis, *day = s->d_axis + nax;
    s->geo.x = axis_view(dax, mx);
    s->geo.y = axis_view(day, my);
    for (int k = 0; k < 4; k++) s->sides.kind[k] = pb.side_kind[k];
    if (!whole) {
        if (L > -G) s->sides.kind[SIDE_W] = BC_INTERFACE;
        if (R < pb.nx + G + 1) s->sides.kind[SIDE_E] = BC_INTERFACE;
        s->sides.col0 = L;
        s->sides.col1 = R;
    }

    s->mixed = pb.precision == SIM_MIXED;
    if (s->mixed) {
        if (cudaMalloc(&s->d_pool32, kPoolArrays * s->nelem * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s->d_axis32, (nax + nay) * sizeof(float)) != cudaSuccess)
            return SIM_ENOMEM;
        carve_levels(s->d_pool32, s->nelem, s->mx.lv, s->mx.w);
        const float *fx = s->d_axis32, *fy = s->d_axis32 + nax;
        s->mx.g.nx = pb.nx;
        s->mx.g.ny = pb.ny;
        s->mx.g.pitch = s->pitch;
        s->mx.g.flag = s->geo.flag;
        s->mx.g.x = axis_view(fx, mx);
        s->mx.g.y = axis_view(fy, my);
        const Coef &k = pb.k;
        s->mx.k = CoefT<float>{(float)k.A, (float)k.B, (float)k.CT1f, (float)k.CT2f, (float)k.CT3f,
                               (float)k.omega, (float)k.dt, (float)k.gx, (float)k.gy, (float)k.hrdt,
                               (float)k.zeta, (float)k.tau, (float)k.B23};
        std::vector<float> a32(nax + nay);
        for (size_t q = 0; q < nax; q++) a32[q] = (float)t.ax[q];
        for (size_t q = 0; q < nay; q++) a32[nax + q] = (float)t.ay[q];
        CUDA_TRY(s, cudaMemcpy(s->d_axis32, a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice));
        CUDA_TRY(s, cudaMemsetAsync(s->mx.w.ru_dy, 0, kWorkArrays * s->nelem * sizeof(float), s->stream));
    }

    s->df = pb.precision == SIM_DF64;
    if (s->df) {
        if (cudaMalloc(&s->d_pooldf, kPoolArrays * s->nelem * sizeof(df64)) != cudaSuccess ||
            cudaMalloc(&s->d_axisdf, (nax + nay) * sizeof(df64)) != cudaSuccess)
            return SIM_ENOMEM;
        carve_levels(s->d_pooldf, s->nelem, s->dfm.lv, s->dfm.w);
        const df64 *fx = s->d_axisdf, *fy = s->d_axisdf + nax;
        s->dfm.g.nx = pb.nx;
        s->dfm.g.ny = pb.ny;
        s->dfm.g.pitch = s->pitch;
        s->dfm.g.flag = s->geo.flag;
        s->dfm.g.x = axis_view(fx, mx);
        s->dfm.g.y = axis_view(fy, my);
        const Coef &k = pb.k;
        s->dfm.k = CoefT<df64>{dfl::split_host(k.A), dfl::split_host(k.B), dfl::split_host(k.CT1f), dfl::split_host(k.CT2f),
                               dfl::split_host(k.CT3f), dfl::split_host(k.omega), dfl::split_host(k.dt), dfl::split_host(k.gx),
                               dfl::split_host(k.gy), dfl::split_host(k.hrdt), dfl::split_host(k.zeta),
                               dfl::split_host(k.tau), dfl::split_host(k.B23)};
        std::vector<df64> adf(nax + nay);
        for (size_t q = 0; q < nax; q++) adf[q] = dfl::split_host(t.ax[q]);
        for (size_t q = 0; q < nay; q++) adf[nax + q] = dfl::split_host(t.ay[q]);
        CUDA_TRY(s, cudaMemcpy(s->d_axisdf, adf.data(), adf.size() * sizeof(df64), cudaMemcpyHostToDevice));
        CUDA_TRY(s, cudaMemsetAsync(s->dfm.w.ru_dy, 0, kWorkArrays * s->nelem * sizeof(df64), s->stream));
    }

    CUDA_TRY(s, cudaMemcpyAsync(s->d_flag, flags->data(), s->nelem * sizeof(uint16_t), cudaMemcpyHostToDevice,
                                s->stream));
    CUDA_TRY(s, cudaMemcpyAsync(s->d_axis, t.ax.data(), nax * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(s, cudaMemcpyAsync(s->d_axis + nax, t.ay.data(), nay * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(s, cudaMemsetAsync(s->work.ru_dy, 0, kWorkArrays * s->nelem * sizeof(double), s->stream));
    CUDA_TRY(s, cudaMemsetAsync(w.res, 0, 4 * sizeof(unsigned long long), s->stream));
    for (int l = 0; l < 3; l++)
        for (int k = 0; k < 6; k++)
            CUDA_TRY(s, cudaMemcpyAsync(level_field(s->lv[l], k), f[k].data(), s->nelem * sizeof(double),
                                        cudaMemcpyHostToDevice, s->stream));
    // from here on the level and scratch pointers are kernel views
    shift_views<double>(s->lv, s->work, s->shift);
    if (s->mixed) shift_views<float>(s->mx.lv, s->mx.w, s->shift);
    if (s->df) shift_views<df64>(s->dfm.lv, s->dfm.w, s->shift);
    for (int l = 0; l < 3; l++) {
        if (whole)
            launch_derive(s->geo, pb.k, s->lv[l], s->stream);
        else
            launch_derive_cols(s->geo, pb.k, s->lv[l], L < 0 ? 0 : L, R, s->stream);
        launch_ghosts(s->geo, s->sides, s->lv[l], false, s->stream);
        if (s->mixed)
            launch_shadow(s->geo, alloc_of(s->lv[l], s->shift), alloc_of(s->mx.lv[l], s->shift), s->nelem,
                          s->stream);
        if (s->df) launch_split(alloc_of(s->lv[l], s->shift), alloc_of(s->dfm.lv[l], s->shift), s->nelem, s->stream);
    }
    if (cudaMalloc(&s->d_inst, sizeof(Inst)) != cudaSuccess || cudaMalloc(&s->d_tiles, sizeof(int)) != cudaSuccess)
        return SIM_ENOMEM;
    CUDA_TRY(s, cudaMemsetAsync(s->d_tiles, 0, sizeof(int), s->stream));
    sim_status st = default_plan(s);
    if (st != SIM_OK) return st;
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

}  // namespace

extern "C" sim_status sim_create(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc, void *stream,
                                 sim_t *out)
{
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    sim_t s = new (std::nothrow) sim_s;
    if (!s) return SIM_ENOMEM;
    sim_status st = read_problem(grid, gas, bc, s->pb, s);
    if (st != SIM_OK) {
        sim_destroy(s);
        return st;
    }
    s->stream = (cudaStream_t)stream;
    Template t;
    make_template(s->pb, t);
    st = build_handle(s, t, -G, s->pb.nx + G + 1);
    if (st != SIM_OK) {
        sim_destroy(s);
        return st;
    }
    *out = s;
    return SIM_OK;
}

extern "C" sim_status sim_step(sim_t s, int n_steps, int scheme)
{
    sim_status st = check_live(s);
    if (st != SIM_OK) return st;
    if (n_steps < 0 || (scheme & ~3)) return fail(s, SIM_EINVAL, "bad n_steps %d or scheme %d", n_steps, scheme);
    const bool implicit = scheme & SIM_IMPLICIT, tvd = scheme & SIM_TVD;
    const Problem &pb = s->pb;
    if (n_steps > 0 && s->df) s->df_dirty = true;
    if (n_steps > 0 && s->mixed) s->mx_dirty = true;

    // Fixed loop-2 length and no event timing: replay one captured graph per
    // step (the three state levels rotate, so a step graph exists for each
    // start level).
    if (pb.tol == 0.0 && !s->timing && !s->graphs_off) {
        for (int step = 0; step < n_steps; step++) {
            sim_s::StepGraph &gr = s->graphs[s->cur][scheme];
            if (!gr.exec) {
                if (!s->cap_stream)
                    CUDA_TRY(s, cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
                cudaGraph_t graph = nullptr;
                CUDA_TRY(s, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
                gr.result = enqueue_step(s, s->cur, implicit, tvd, s->cap_stream, gr.counts);
                CUDA_TRY(s, cudaStreamEndCapture(s->cap_stream, &graph));
                cudaError_t e = cudaGraphInstantiate(&gr.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) {
                    gr.exec = nullptr;
                    return fail(s, SIM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
                }
            }
            CUDA_TRY(s, cudaGraphLaunch(gr.exec, s->stream));
            for (int k = 0; k < SIM_K_COUNT; k++) s->launches[k] += gr.counts[k];
            s->cur = gr.result;
            s->last_iters = pb.iters;
        }
        CUDA_TRY(s, cudaGetLastError());
        return SIM_OK;
    }

    for (int step = 0; step < n_steps; step++) {
        const int prev = s->cur;
        if (pb.tol == 0.0) {
            s->cur = enqueue_step(s, prev, implicit, tvd, s->stream, nullptr);
            s->last_iters = pb.iters;
            continue;
        }
        // loop 2 until every residual <= tol: one iteration at a time, reading
        // the residuals back after each (Section 5: the only per-iteration
        // device-to-host traffic)
        int old = prev, it = 0;
        if (!implicit) enqueue_explicit(s, prev, tvd, s->stream, nullptr);
        for (it = 1; it <= pb.iters; it++) {
            old = enqueue_iteration(s, prev, old, implicit, tvd, !implicit && it == 1, s->stream, nullptr);
            CUDA_TRY(s, cudaMemcpyAsync(s->h_res, s->work.res, 4 * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s->stream));
            CUDA_TRY(s, cudaStreamSynchronize(s->stream));
            double mx = 0.0;
            bool bad = false;
            for (int q = 0; q < 4; q++) {
                double r;
                std::memcpy(&r, &s->h_res[q], sizeof r);
                if (!std::isfinite(r)) bad = true;
                mx = std::fmax(mx, r);
            }
            if (bad) {
                s->cur = old;
                s->last_iters = it;
                s->diverged = true;
                s->set_mask = 0;
                return fail(s, SIM_EDIVERGED, "non-finite residual in step %d, iteration %d", step, it);
            }
            if (mx <= pb.tol) break;
        }
        s->last_iters = it > pb.iters ? pb.iters : it;
        s->cur = old;
    }
    CUDA_TRY(s, cudaGetLastError());
    return SIM_OK;
}

extern "C" sim_status sim_fields(sim_t s, int field, double *host_dst, size_t n)
{
    if (!s) return SIM_EINVAL;
    if (field < 0 || field > 5 || !host_dst) return fail(s, SIM_EINVAL, "bad field %d or null destination", field);
    const size_t need = field_count(s->pb, field);
    if (n != need) return fail(s, SIM_EINVAL, "field %d has %zu elements, got %zu", field, need, n);
    sync_out(s);
    launch_gather(s->geo, field, s->lv[s->cur], s->d_stage, s->stream);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaMemcpyAsync(host_dst, s->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

extern "C" sim_status sim_field_ptr(sim_t s, int field, void **dev, size_t *pitch)
{
    if (!s) return SIM_EINVAL;
    if (field < 0 || field > 5 || !dev || !pitch) return fail(s, SIM_EINVAL, "bad field %d or null output", field);
    sync_out(s);
    *dev = level_field(s->lv[s->cur], field) + (size_t)G * s->pitch + G;
    *pitch = (size_t)s->pitch;
    return SIM_OK;
}

extern "C" sim_status sim_set_fields(sim_t s, int field, const double *host_src, size_t n)
{
    if (!s) return SIM_EINVAL;
    if (field < 0 || field > 3 || !host_src) return fail(s, SIM_EINVAL, "only u, v, p, T can be set (field %d)", field);
    const size_t need = field_count(s->pb, field);
    if (n != need) return fail(s, SIM_EINVAL, "field %d has %zu elements, got %zu", field, need, n);
    for (size_t q = 0; q < n; q++)
        if (!std::isfinite(host_src[q]) || ((field == SIM_FIELD_T || field == SIM_FIELD_P) && !(host_src[q] > 0.0)))
            return fail(s, SIM_EINVAL, "field %d: value %zu is not admissible", field, q);
    sync_out(s);
    const Level &L = s->lv[s->cur];
    CUDA_TRY(s, cudaMemcpyAsync(s->d_stage, host_src, n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    launch_scatter(s->geo, field, s->d_stage, L, s->stream);
    launch_derive(s->geo, s->pb.k, L, s->stream);
    launch_ghosts(s->geo, s->sides, L, false, s->stream);
    if (s->mixed) launch_shadow(s->geo, L, s->mx.lv[s->cur], s->nelem, s->stream);
    if (s->df) launch_split(L, s->dfm.lv[s->cur], s->nelem, s->stream);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    if (s->diverged) {
        s->set_mask |= 1u << field;
        if (s->set_mask == 0xFu) {
            s->diverged = false;
            s->set_mask = 0;
        }
    }
    return SIM_OK;
}

namespace {

// Residual words -> doubles; false if one is not finite.
bool read_residuals(const unsigned long long *bits, double out[4])
{
    bool ok = true;
    for (int q = 0; q < 4; q++) {
        std::memcpy(&out[q], &bits[q], sizeof(double));
        if (!std::isfinite(out[q])) ok = false;
    }
    return ok;
}

// Device address of a host array of `bytes` bytes when its first and last
// bytes lie in page-locked memory that the device addresses, mapped as one
// range; nullptr otherwise (pageable memory, or memory CUDA does not know),
// and the caller copies with cudaMemcpyAsync instead.
const void *mapped_view(const void *p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *last = (const char *)p + (bytes - 1);
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost || !b.devicePointer ||
        (const char *)b.devicePointer - (const char *)a.devicePointer != (std::ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

sim_status ensure_state_stage(sim_t s)
{
    if (s->d_state) return SIM_OK;
    const size_t n = 4 * (size_t)(s->pb.nx + 1) * (s->pb.ny + 1);
    if (cudaMalloc(&s->d_state, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&s->d_bad, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&s->h_bad, sizeof(unsigned)) != cudaSuccess) {
        cudaFree(s->d_state);
        cudaFree(s->d_bad);
        s->d_state = nullptr;
        s->d_bad = nullptr;
        return fail(s, SIM_ENOMEM, "no memory for the state staging area");
    }
    return SIM_OK;
}

}  // namespace

extern "C" sim_status sim_set_state(sim_t s, const double *u, const double *v, const double *p, const double *T)
{
    if (!s) return SIM_EINVAL;
    if (!u || !v || !p || !T) return fail(s, SIM_EINVAL, "null state array");
    sim_status st = ensure_state_stage(s);
    if (st != SIM_OK) return st;
    const size_t nu = field_count(s->pb, SIM_FIELD_U), nv = field_count(s->pb, SIM_FIELD_V);
    const size_t nc = field_count(s->pb, SIM_FIELD_P);
    const double *src[4] = {u, v, p, T};
    const size_t off[4] = {0, nu, nu + nv, nu + nv + nc}, cnt[4] = {nu, nv, nc, nc};
    CUDA_TRY(s, cudaMemsetAsync(s->d_bad, 0, sizeof(unsigned), s->stream));
    // page-locked arrays: one kernel reads them over the host link, stages and
    // checks them; otherwise four copies and the check
    StateSrc view{};
    bool mapped = true;
    for (int f = 0; f < 4 && mapped; f++) {
        view.f[f] = (const double *)mapped_view(src[f], cnt[f] * sizeof(double));
        mapped = view.f[f] != nullptr;
    }
    if (mapped) {
        launch_stage_state(view, nu, nv, nc, s->d_state, s->d_bad, s->stream);
    } else {
        for (int f = 0; f < 4; f++)
            CUDA_TRY(s, cudaMemcpyAsync(s->d_state + off[f], src[f], cnt[f] * sizeof(double),
                                        cudaMemcpyHostToDevice, s->stream));
        launch_validate_state(s->d_state, nu, nv, nc, s->d_bad, s->stream);
    }
    CUDA_TRY(s, cudaMemcpyAsync(s->h_bad, s->d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    if (*s->h_bad) return fail(s, SIM_EINVAL, "state not admissible (non-finite value, or p or T <= 0)");
    // every unknown is overwritten: the FP64 level needs no refresh from the
    // double-float one first
    const Level &L = s->lv[s->cur];
    launch_scatter_state(s->geo, s->pb.k, s->d_state, L, s->stream);
    launch_ghosts(s->geo, s->sides, L, false, s->stream);
    if (s->mixed) launch_shadow(s->geo, L, s->mx.lv[s->cur], s->nelem, s->stream);
    if (s->df) launch_split(L, s->dfm.lv[s->cur], s->nelem, s->stream);
    s->df_dirty = false;
    s->mx_dirty = false;
    CUDA_TRY(s, cudaGetLastError());
    s->diverged = false;
    s->set_mask = 0;
    return SIM_OK;
}

extern "C" sim_status sim_get_state(sim_t s, double *u, double *v, double *p, double *T, double res[4])
{
    if (!s) return SIM_EINVAL;
    if (!u || !v || !p || !T) return fail(s, SIM_EINVAL, "null state array");
    sim_status st = ensure_state_stage(s);
    if (st != SIM_OK) return st;
    const size_t nu = field_count(s->pb, SIM_FIELD_U), nv = field_count(s->pb, SIM_FIELD_V);
    const size_t nc = field_count(s->pb, SIM_FIELD_P);
    double *dst[4] = {u, v, p, T};
    const size_t off[4] = {0, nu, nu + nv, nu + nv + nc}, cnt[4] = {nu, nv, nc, nc};
    sync_out(s);
    // page-locked arrays: the gather kernel writes them over the host link;
    // otherwise it writes the staging array, copied out field by field
    StatePtrs view{}, stage{};
    bool mapped = true;
    for (int f = 0; f < 4 && mapped; f++) {
        view.f[f] = (double *)mapped_view(dst[f], cnt[f] * sizeof(double));
        mapped = view.f[f] != nullptr;
    }
    for (int f = 0; f < 4; f++) stage.f[f] = s->d_state + off[f];
    launch_gather_state(s->geo, s->lv[s->cur], mapped ? view : stage, s->stream);
    CUDA_TRY(s, cudaGetLastError());
    if (!mapped)
        for (int f = 0; f < 4; f++)
            CUDA_TRY(s, cudaMemcpyAsync(dst[f], s->d_state + off[f], cnt[f] * sizeof(double),
                                        cudaMemcpyDeviceToHost, s->stream));
    if (res)
        CUDA_TRY(s, cudaMemcpyAsync(s->h_res, s->work.res, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    if (res && !read_residuals(s->h_res, res)) {
        s->diverged = true;
        s->set_mask = 0;
        return fail(s, SIM_EDIVERGED, "non-finite residual");
    }
    return SIM_OK;
}

extern "C" sim_status sim_residuals(sim_t s, double out[4], int *iters_last_step)
{
    if (!s || !out) return SIM_EINVAL;
    CUDA_TRY(s, cudaMemcpyAsync(s->h_res, s->work.res, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    bool bad = false;
    for (int q = 0; q < 4; q++) {
        std::memcpy(&out[q], &s->h_res[q], sizeof(double));
        if (!std::isfinite(out[q])) bad = true;
    }
    if (iters_last_step) *iters_last_step = s->last_iters;
    if (bad) {
        s->diverged = true;
        s->set_mask = 0;
        return fail(s, SIM_EDIVERGED, "non-finite residual");
    }
    return SIM_OK;
}

extern "C" sim_status sim_coefficients(sim_t s, double out[9])
{
    if (!s || !out) return SIM_EINVAL;
    const Coef &k = s->pb.k;
    out[0] = k.A; out[1] = k.B; out[2] = k.CT1f; out[3] = k.CT2f; out[4] = k.CT3f;
    out[5] = k.omega; out[6] = s->pb.u_in; out[7] = k.dt; out[8] = (double)s->pb.nx * s->pb.ny;
    return SIM_OK;
}

extern "C" sim_status sim_set_plan(sim_t s, int tile_x, int tile_y, int ctas, int asm_ctas)
{
    if (!s) return SIM_EINVAL;
    if (!plan_shape_ok(tile_x, tile_y, ctas) || asm_ctas < 0)
        return fail(s, SIM_EINVAL,
                    "tile %d x %d with %d / %d CTAs: want 32, 64, 128 or 256 threads, tile x in {16, ..., 256}, "
                    "CTAs >= 0", tile_x, tile_y, ctas, asm_ctas);
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    sim_status st = single_plan(s, tile_x, tile_y, ctas, asm_ctas);
    if (st != SIM_OK) return st;
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

extern "C" sim_status sim_profile(sim_t s, int enable)
{
    if (!s) return SIM_EINVAL;
    if (enable) {
        CUDA_TRY(s, cudaStreamSynchronize(s->stream));
        for (auto &m : s->marks) {
            s->spare.push_back(m.e0);
            s->spare.push_back(m.e1);
        }
        s->marks.clear();
        for (auto &c : s->launches) c = 0;
    }
    s->timing = enable == 1;
    return SIM_OK;
}

extern "C" sim_status sim_profile_read(sim_t s, int cls, double *ms, long long *launches)
{
    if (!s || cls < 0 || cls >= SIM_K_COUNT || !ms || !launches) return SIM_EINVAL;
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    double total = 0.0;
    for (auto &m : s->marks)
        if (m.cls == cls) {
            float t = 0.f;
            CUDA_TRY(s, cudaEventElapsedTime(&t, m.e0, m.e1));
            total += t;
        }
    *ms = total;
    *launches = s->launches[cls];
    return SIM_OK;
}

extern "C" const char *sim_last_error(sim_t s)
{
    return s ? s->err : "null handle";
}

extern "C" void sim_destroy(sim_t s)
{
    if (!s) return;
    if (s->d_pool) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_pool);
    cudaFree(s->d_flag);
    cudaFree(s->d_axis);
    cudaFree(s->d_stage);
    cudaFree(s->d_state);
    cudaFree(s->d_bad);
    if (s->h_bad) cudaFreeHost(s->h_bad);
    cudaFree(s->work.res);
    cudaFree(s->d_pool32);
    cudaFree(s->d_axis32);
    cudaFree(s->d_inst);
    cudaFree(s->d_tiles);
    cudaFree(s->d_pooldf);
    cudaFree(s->d_axisdf);
    if (s->h_res) cudaFreeHost(s->h_res);
    for (auto &m : s->marks) {
        cudaEventDestroy(m.e0);
        cudaEventDestroy(m.e1);
    }
    for (auto e : s->spare) cudaEventDestroy(e);
    for (auto &row : s->graphs)
        for (auto &g : row)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

// ==================================================================== batches

struct sim_batch_s {
    std::vector<sim_t> inst;
    cudaStream_t stream = nullptr;
    bool mixed = false;
    int prec = PREC_FP64;
    int iters = 1;
    Inst *d_inst = nullptr;
    int *d_tiles = nullptr;
    size_t tiles_cap = 0;
    BatchPlan plan{};
    bool ghosts = false;                      // some problem has a symmetry side
    // persistent step: one cooperative kernel per time step (persistent.cu),
    // captured with the reset of its barrier in the step's CUDA graph, or
    // launched directly if the capture is refused (persistent_direct)
    bool persistent = false;
    bool persistent_direct = false;
    GridBarrier *d_bar = nullptr;
    unsigned *h_err = nullptr;                // pinned copy of the barrier's error word
    struct Graph { cudaGraphExec_t exec = nullptr; int result = 0; };
    Graph graphs[3][4];
    cudaStream_t cap_stream = nullptr;
    int cur = 0;
    char err[256] = {0};
};

namespace {

sim_status batch_barrier_status(sim_batch_t b);

sim_status bfail(sim_batch_t b, sim_status st, const char *fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof b->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define BCUDA_TRY(b, call)                                                          \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return bfail(b, SIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

void drop_graphs(sim_batch_t b)
{
    for (auto &row : b->graphs)
        for (auto &g : row)
            if (g.exec) {
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
            }
}

// Tile list for a tile shape: every problem's (nx+1) x (ny+1) positions cut
// into tx x ty tiles; `grid` resident CTAs walk the list.
sim_status plan_tiles(sim_batch_t b, int tx, int ty, int grid)
{
    std::vector<Inst> host(b->inst.size());
    std::vector<int> tiles;
    for (size_t q = 0; q < b->inst.size(); q++) {
        const sim_t s = b->inst[q];
        host[q] = inst_of(s, tx, (int)tiles.size());
        tiles.insert(tiles.end(), (size_t)tiles_of(s, tx, ty), (int)q);
    }
    if (!b->d_inst)
        BCUDA_TRY(b, cudaMalloc(&b->d_inst, host.size() * sizeof(Inst)));
    if (tiles.size() > b->tiles_cap) {
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        BCUDA_TRY(b, cudaMalloc(&b->d_tiles, tiles.size() * sizeof(int)));
        b->tiles_cap = tiles.size();
    }
    BCUDA_TRY(b, cudaMemcpyAsync(b->d_inst, host.data(), host.size() * sizeof(Inst), cudaMemcpyHostToDevice, b->stream));
    BCUDA_TRY(b, cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    // one CTA per tile (a count of CTAs at least the tiles' is the same): the
    // mixed path's FP32 assembly walks the tiles with its resident CTAs
    // instead (as for a single problem, default_plan)
    if (grid >= (int)tiles.size()) grid = 0;
    int grid_asm = 0;
    if (grid == 0 && b->prec == PREC_MIXED) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            grid_asm = std::min((int)tiles.size(), 1024 / (tx * ty) * sms);
    }
    b->plan = BatchPlan{b->d_inst, b->d_tiles, (int)host.size(), (int)tiles.size(), tx, ty,
                        grid > 0 ? std::min(grid, (int)tiles.size()) : (int)tiles.size(), host[0], grid_asm};
    drop_graphs(b);
    return SIM_OK;
}

// The phases of one time step from level `prev` for the persistent kernel,
// in the order the per-phase launches take; returns the result level.
int step_phases(sim_batch_t b, int prev, bool implicit, bool tvd, PhaseList &ph)
{
    ph.n = 0;
    auto add = [&](int kind, int a, int bb, int c) {
        ph.kind[ph.n] = (unsigned char)kind;
        ph.a[ph.n] = (unsigned char)a;
        ph.b[ph.n] = (unsigned char)bb;
        ph.c[ph.n] = (unsigned char)c;
        ph.n++;
    };
    if (!implicit) {
        add(PH_FACES, prev, tvd ? 1 : 0, 0);
        add(PH_EXPLICIT, prev, 0, 0);
    }
    int old = prev;
    for (int it = 1; it <= b->iters; it++) {
        int nw = (old + 1) % 3;
        if (nw == prev) nw = (nw + 1) % 3;
        if (implicit || it > 1) add(PH_FACES, old, (tvd && implicit) ? 1 : 0, 0);
        add(PH_ASSEMBLE, prev, old, nw);
        add(PH_PRESSURE, prev, old, nw);
        add(PH_VELOCITY, old, nw, 0);
        old = nw;
    }
    return old;
}

// One time step of every problem from level `prev`; returns the result level
// (-1 if the persistent kernel could not be launched).
int enqueue_batch_step(sim_batch_t b, int prev, bool implicit, bool tvd, cudaStream_t st)
{
    const BatchPlan &bp = b->plan;
    if (b->persistent) {
        PhaseList ph{};
        const int result = step_phases(b, prev, implicit, tvd, ph);
        const int ctas = std::min(persistent_ctas(b->prec, implicit, tvd, bp.tx * bp.ty), bp.n_tiles);
        if (ctas < 1 || launch_step_persistent(bp, ph, b->d_bar, b->prec, implicit, tvd, ctas, st) != cudaSuccess)
            return -1;
        return result;
    }
    if (!implicit) {
        launch_faces(bp, b->prec, prev, tvd, true, st);
        launch_explicit(bp, b->prec, prev, tvd, st);
    }
    int old = prev;
    for (int it = 1; it <= b->iters; it++) {
        int nw = (old + 1) % 3;
        if (nw == prev) nw = (nw + 1) % 3;
        if (implicit || it > 1)         // an explicit step's first iteration reuses the faces of n-1
            launch_faces(bp, b->prec, old, tvd, implicit, st);
        launch_assemble(bp, b->prec, prev, old, nw, implicit, tvd, st);
        launch_pressure(bp, b->prec, prev, old, nw, st);
        launch_velocity(bp, b->prec, old, nw, st);
        if (b->ghosts)
            for (sim_t s : b->inst)
                if (ghost_kernels(s->sides, true)) {
                    if (s->df) {
                        launch_ghosts_df(s->dfm, s->sides, nw, true, st);
                    } else {
                        launch_ghosts(s->geo, s->sides, s->lv[nw], true, st);
                        if (b->mixed) launch_ghosts_f32(s->mx, s->sides, nw, true, st);
                    }
                }
        old = nw;
    }
    return old;
}

void set_levels(sim_batch_t b, int cur)
{
    b->cur = cur;
    for (sim_t s : b->inst) {
        s->cur = cur;
        s->last_iters = b->iters;
        if (s->df) s->df_dirty = true;
        if (s->mixed) s->mx_dirty = true;
    }
}

}  // namespace

extern "C" sim_status sim_batch_create(int n, const sim_grid *grids, const sim_gas *gases, const sim_bc *bcs,
                                       void *stream, sim_batch_t *out)
{
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    if (n < 1 || !grids || !gases || !bcs) return SIM_EINVAL;
    for (int q = 0; q < n; q++) {
        if (bcs[q].precision != bcs[0].precision || bcs[q].iters != bcs[0].iters || bcs[q].tol != 0.0)
            return SIM_EINVAL;
    }
    sim_batch_t b = new (std::nothrow) sim_batch_s;
    if (!b) return SIM_ENOMEM;
    b->stream = (cudaStream_t)stream;
    b->mixed = bcs[0].precision == SIM_MIXED;
    b->prec = b->mixed ? PREC_MIXED : bcs[0].precision == SIM_DF64 ? PREC_DF64 : PREC_FP64;
    b->iters = bcs[0].iters;
    for (int q = 0; q < n; q++) {
        sim_t s = nullptr;
        sim_status st = sim_create(&grids[q], &gases[q], &bcs[q], stream, &s);
        if (st != SIM_OK) {
            sim_batch_destroy(b);
            return st;
        }
        b->inst.push_back(s);
        if (ghost_kernels(s->sides, true)) b->ghosts = true;
    }
    sim_status st = plan_tiles(b, 32, 8, 0);
    if (st != SIM_OK) {
        sim_batch_destroy(b);
        return st;
    }
    *out = b;
    return SIM_OK;
}

extern "C" sim_status sim_batch_step(sim_batch_t b, int n_steps, int scheme)
{
    if (!b) return SIM_EINVAL;
    if (n_steps < 0 || (scheme & ~3)) return bfail(b, SIM_EINVAL, "bad n_steps %d or scheme %d", n_steps, scheme);
    const bool implicit = scheme & SIM_IMPLICIT, tvd = scheme & SIM_TVD;
    for (int step = 0; step < n_steps; step++) {
        if (b->persistent && b->persistent_direct) {      // one cooperative launch per step
            const int result = enqueue_batch_step(b, b->cur, implicit, tvd, b->stream);
            if (result < 0) return bfail(b, SIM_ECUDA, "persistent step launch failed: %s",
                                         cudaGetErrorString(cudaGetLastError()));
            set_levels(b, result);
            continue;
        }
        sim_batch_s::Graph &g = b->graphs[b->cur][scheme];
        if (!g.exec) {
            if (!b->cap_stream)
                BCUDA_TRY(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            BCUDA_TRY(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            g.result = enqueue_batch_step(b, b->cur, implicit, tvd, b->cap_stream);
            const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &graph);
            if (g.result < 0 || ec != cudaSuccess) {
                // the persistent step's cooperative launch was not captured:
                // launch it directly from now on
                if (graph) cudaGraphDestroy(graph);
                const cudaError_t why = ec != cudaSuccess ? ec : cudaGetLastError();
                cudaGetLastError();
                if (!b->persistent)
                    return bfail(b, SIM_ECUDA, "step capture failed: %s", cudaGetErrorString(why));
                b->persistent_direct = true;
                step--;
                continue;
            }
            cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                g.exec = nullptr;
                return bfail(b, SIM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            }
        }
        BCUDA_TRY(b, cudaGraphLaunch(g.exec, b->stream));
        set_levels(b, g.result);
    }
    BCUDA_TRY(b, cudaGetLastError());
    return SIM_OK;
}

namespace {

// SIM_ETIMEOUT if a grid barrier of the persistent step ran out of time since
// the barrier was last cleared (the results of that step are not valid).
sim_status batch_barrier_status(sim_batch_t b)
{
    if (!b->d_bar) return SIM_OK;
    BCUDA_TRY(b, cudaMemcpyAsync(b->h_err, &b->d_bar->err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    if (*b->h_err) return bfail(b, SIM_ETIMEOUT, "a grid barrier of the persistent step timed out");
    return SIM_OK;
}

}  // namespace

extern "C" sim_status sim_batch_fields(sim_batch_t b, int instance, int field, double *host_dst, size_t n)
{
    if (!b || instance < 0 || instance >= (int)b->inst.size()) return SIM_EINVAL;
    sim_status st = batch_barrier_status(b);
    if (st != SIM_OK) return st;
    return sim_fields(b->inst[instance], field, host_dst, n);
}

extern "C" sim_status sim_batch_residuals(sim_batch_t b, int instance, double out[4])
{
    if (!b || instance < 0 || instance >= (int)b->inst.size()) return SIM_EINVAL;
    sim_status st = batch_barrier_status(b);
    if (st != SIM_OK) return st;
    return sim_residuals(b->inst[instance], out, nullptr);
}

extern "C" sim_status sim_batch_set_persistent(sim_batch_t b, int on)
{
    if (!b) return SIM_EINVAL;
    if (on && b->ghosts)
        return bfail(b, SIM_EINVAL, "the persistent step does not run the ghost kernels of symmetry sides");
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    if (on && !b->d_bar) {
        if (cudaMalloc(&b->d_bar, sizeof(GridBarrier)) != cudaSuccess ||
            cudaMallocHost(&b->h_err, sizeof(unsigned)) != cudaSuccess)
            return bfail(b, SIM_ENOMEM, "no memory for the grid barrier");
        BCUDA_TRY(b, cudaMemset(b->d_bar, 0, sizeof(GridBarrier)));
    }
    b->persistent = on != 0;
    b->persistent_direct = false;
    drop_graphs(b);
    return SIM_OK;
}

extern "C" sim_status sim_batch_plan_info(sim_batch_t b, int out[4])
{
    if (!b || !out) return SIM_EINVAL;
    out[0] = b->plan.tx;
    out[1] = b->plan.ty;
    out[2] = b->plan.grid;
    out[3] = b->persistent ? (b->persistent_direct ? 2 : 1) : 0;
    return SIM_OK;
}

namespace {

// Autotuner of sim_batch_tune: every tile shape x CTA count of the candidate
// lists, each timed over three steps after one warm-up step from the same
// saved state.
sim_status tune_batch(sim_batch_t b, int scheme, int out[3])
{
    const bool implicit = scheme & SIM_IMPLICIT, tvd = scheme & SIM_TVD;
    // keep a copy of every problem's current level (FP64 and FP32 shadow) and
    // residual words, so that tuning leaves the simulation where it was
    size_t total = 0;
    const size_t shadow = b->mixed ? sizeof(float) : b->prec == PREC_DF64 ? sizeof(df64) : 0;
    for (sim_t s : b->inst) total += 6 * s->nelem * (sizeof(double) + shadow) + 32;
    unsigned char *save = nullptr;
    if (cudaMalloc(&save, total) != cudaSuccess) return bfail(b, SIM_ENOMEM, "no memory for the tuning copy");
    const int start = b->cur;
    auto copy_state = [&](bool to_save) -> cudaError_t {
        unsigned char *p = save;
        for (sim_t s : b->inst) {
            const size_t n64 = s->nelem * sizeof(double), n32 = s->nelem * sizeof(float);
            for (int f = 0; f < 6; f++) {
                double *lvf = level_field(s->lv[start], f);
                cudaError_t e = to_save ? cudaMemcpyAsync(p, lvf, n64, cudaMemcpyDeviceToDevice, b->stream)
                                        : cudaMemcpyAsync(lvf, p, n64, cudaMemcpyDeviceToDevice, b->stream);
                if (e != cudaSuccess) return e;
                p += n64;
                if (b->mixed) {
                    const LevelT<float> &L = s->mx.lv[start];
                    float *f32 = f == 0 ? L.u : f == 1 ? L.v : f == 2 ? L.p : f == 3 ? L.T : f == 4 ? L.rho : L.gam;
                    e = to_save ? cudaMemcpyAsync(p, f32, n32, cudaMemcpyDeviceToDevice, b->stream)
                                : cudaMemcpyAsync(f32, p, n32, cudaMemcpyDeviceToDevice, b->stream);
                    if (e != cudaSuccess) return e;
                    p += n32;
                }
                if (b->prec == PREC_DF64) {
                    const LevelT<df64> &L = s->dfm.lv[start];
                    df64 *fd = f == 0 ? L.u : f == 1 ? L.v : f == 2 ? L.p : f == 3 ? L.T : f == 4 ? L.rho : L.gam;
                    const size_t nd = s->nelem * sizeof(df64);
                    e = to_save ? cudaMemcpyAsync(p, fd, nd, cudaMemcpyDeviceToDevice, b->stream)
                                : cudaMemcpyAsync(fd, p, nd, cudaMemcpyDeviceToDevice, b->stream);
                    if (e != cudaSuccess) return e;
                    p += nd;
                }
            }
            cudaError_t e = to_save ? cudaMemcpyAsync(p, s->work.res, 32, cudaMemcpyDeviceToDevice, b->stream)
                                    : cudaMemcpyAsync(s->work.res, p, 32, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            p += 32;
        }
        return cudaSuccess;
    };
    if (copy_state(true) != cudaSuccess) {
        cudaFree(save);
        return bfail(b, SIM_ECUDA, "saving the state before tuning failed");
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int shapes[6][2] = {{32, 8}, {64, 4}, {128, 2}, {16, 16}, {32, 4}, {64, 2}};
    // CTA counts: 2 or 4 per SM walking the tiles, one CTA per tile (0), and
    // the persistent step kernel (-1; not with symmetry sides)
    const int grids[4] = {2 * sms, 4 * sms, 0, -1};
    const int n_grids = b->ghosts ? 3 : 4;
    if (!b->ghosts && sim_batch_set_persistent(b, 0) != SIM_OK) {
        cudaFree(save);
        return SIM_ECUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bx = 32, by = 8, bg = 0;
    bool bpers = false;
    sim_status st = SIM_OK;
    for (auto &sh : shapes) {
        for (int gi = 0; gi < n_grids; gi++) {
            const int gsz = grids[gi];
            if ((st = plan_tiles(b, sh[0], sh[1], gsz < 0 ? 0 : gsz)) != SIM_OK) break;
            b->persistent = gsz < 0;
            if (b->persistent && (st = sim_batch_set_persistent(b, 1)) != SIM_OK) break;
            int lv = start;
            bool ok = (lv = enqueue_batch_step(b, lv, implicit, tvd, b->stream)) >= 0;     // warm-up
            cudaEventRecord(e0, b->stream);
            for (int r = 0; r < 3 && ok; r++) ok = (lv = enqueue_batch_step(b, lv, implicit, tvd, b->stream)) >= 0;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = bfail(b, SIM_ECUDA, "tuning run failed");
                break;
            }
            if (b->persistent && ok) ok = batch_barrier_status(b) == SIM_OK;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ok && ms < best) {
                best = ms;
                bx = sh[0];
                by = sh[1];
                bg = gsz < 0 ? 0 : gsz;
                bpers = gsz < 0;
            }
            // next candidate starts from the saved state again
            if (copy_state(false) != cudaSuccess) {
                st = bfail(b, SIM_ECUDA, "restoring the state failed");
                break;
            }
        }
        if (st != SIM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(b->stream);
    cudaFree(save);
    b->persistent = false;
    if (st != SIM_OK) return st;
    set_levels(b, start);
    if ((st = plan_tiles(b, bx, by, bg)) != SIM_OK) return st;
    if (bpers && (st = sim_batch_set_persistent(b, 1)) != SIM_OK) return st;
    out[0] = bx;
    out[1] = by;
    out[2] = b->plan.grid;
    return SIM_OK;
}

}  // namespace

extern "C" sim_status sim_batch_tune(sim_batch_t b, int scheme, int out[3])
{
    if (!b || !out || (scheme & ~3)) return SIM_EINVAL;
    return tune_batch(b, scheme, out);
}

extern "C" sim_status sim_batch_set_tiles(sim_batch_t b, int tx, int ty, int ctas)
{
    if (!b) return SIM_EINVAL;
    if (!plan_shape_ok(tx, ty, ctas))
        return bfail(b, SIM_EINVAL,
                     "tile %d x %d with %d CTAs: want 32, 64, 128 or 256 threads, tile x in {16, ..., 256}, CTAs >= 0",
                     tx, ty, ctas);
    BCUDA_TRY(b, cudaStreamSynchronize(b->stream));
    return plan_tiles(b, tx, ty, ctas);
}

extern "C" const char *sim_batch_last_error(sim_batch_t b)
{
    return b ? b->err : "null batch";
}

extern "C" void sim_batch_destroy(sim_batch_t b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_inst);
    cudaFree(b->d_tiles);
    cudaFree(b->d_bar);
    if (b->h_err) cudaFreeHost(b->h_err);
    for (sim_t s : b->inst) sim_destroy(s);
    delete b;
}

// =================================================================== x-strips

struct sim_strips_s {
    Problem pb;
    std::vector<sim_t> strip;                 // one windowed handle per strip
    std::vector<int> own0, own1;              // owned cell columns [own0, own1)
    cudaStream_t stream = nullptr;
    HaloCopy *d_copies = nullptr;             // 3 x n_copies: the halo copies of each level
    int n_copies = 0, max_words = 0;
    double *d_stage = nullptr;                // logical-shape staging array of the whole problem
    unsigned long long *h_res = nullptr;      // pinned: 4 residual words per strip
    struct Graph { cudaGraphExec_t exec = nullptr; int result = 0; };
    Graph graphs[3][4];
    cudaStream_t cap_stream = nullptr;
    int cur = 0;
    char err[256] = {0};
};

namespace {

// Columns of a halo: the strips exchange this many columns of every field on
// each side once per loop-2 iteration.  A position's face quantities read the
// previous iterate two columns away, the assembly reads face quantities one
// column away, the pressure reads the assembly's d and u^ one column east and
// the velocity correction the pressure one column west: the owned columns'
// new values need the previous iterate four columns beyond them.
constexpr int kStripHalo = 4;
constexpr int kMaxStrips = 64;

// Strip k of n over nx cells: owned columns [a, b) (nearly equal widths of at
// least two halos), computed positions [c0, c1) = [a - halo rounded down to a
// multiple of 32 (the warps keep the whole problem's 32-wide row segments),
// b + halo) clipped to [0, nx + 1), stored columns [c0 - 2, c1 + 2).
bool strip_layout(int nx, int n, int k, int out[6])
{
    if (n < 1 || n > kMaxStrips || k < 0 || k >= n || nx < 2 * kStripHalo * n) return false;
    const int a = (int)((long long)k * nx / n), b = (int)((long long)(k + 1) * nx / n);
    int c0 = a - kStripHalo;
    if (c0 < 0) c0 = 0;
    c0 = c0 / 32 * 32;
    const int c1 = k == n - 1 ? nx + 1 : b + kStripHalo;
    out[0] = a;
    out[1] = b;
    out[2] = c0 - G;
    out[3] = c1 + G;
    out[4] = c0;
    out[5] = c1;
    return true;
}

sim_status sfail(sim_strips_t h, sim_status st, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define SCUDA_TRY(h, call)                                                          \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return sfail(h, SIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

// The device arrays (kernel views) of level l that carry the state of the
// strip's arithmetic, with their element sizes.
int level_arrays(const sim_s *s, int l, void *ptr[12], int bytes[12])
{
    int n = 0;
    auto add6 = [&](void *u, void *v, void *p, void *T, void *rho, void *gam, int b) {
        void *a[6] = {u, v, p, T, rho, gam};
        for (void *x : a) {
            ptr[n] = x;
            bytes[n++] = b;
        }
    };
    if (s->df) {
        const LevelT<df64> &L = s->dfm.lv[l];
        add6(L.u, L.v, L.p, L.T, L.rho, L.gam, (int)sizeof(df64));
    } else {
        const Level &L = s->lv[l];
        add6(L.u, L.v, L.p, L.T, L.rho, L.gam, (int)sizeof(double));
        if (s->mixed) {
            const LevelT<float> &M = s->mx.lv[l];
            add6(M.u, M.v, M.p, M.T, M.rho, M.gam, (int)sizeof(float));
        }
    }
    return n;
}

// One time step of every strip from level `prev`: the explicit terms (explicit
// scheme), then per loop-2 iteration each strip's four kernels and ghost
// refresh, then one launch that copies every halo of the new level from the
// strip owning it.  Returns the result level.
int enqueue_strips_step(sim_strips_t h, int prev, bool implicit, bool tvd, cudaStream_t st)
{
    long long counts[SIM_K_COUNT] = {0};
    if (!implicit)
        for (sim_t s : h->strip) enqueue_explicit(s, prev, tvd, st, counts);
    int old = prev;
    for (int it = 1; it <= h->pb.iters; it++) {
        int nw = old;
        for (sim_t s : h->strip) nw = enqueue_iteration(s, prev, old, implicit, tvd, !implicit && it == 1, st, counts);
        launch_halo_copies(h->d_copies + (size_t)nw * h->n_copies, h->n_copies, h->max_words, st);
        old = nw;
    }
    return old;
}

}  // namespace

extern "C" sim_status sim_strips_layout(int nx, int n_strips, int strip, int out[6])
{
    if (!out || !strip_layout(nx, n_strips, strip, out)) return SIM_EINVAL;
    return SIM_OK;
}

extern "C" sim_status sim_strips_create(const sim_grid *grid, const sim_gas *gas, const sim_bc *bc, int n_strips,
                                        void *stream, sim_strips_t *out)
{
    if (!out) return SIM_EINVAL;
    *out = nullptr;
    sim_strips_t h = new (std::nothrow) sim_strips_s;
    if (!h) return SIM_ENOMEM;
    h->stream = (cudaStream_t)stream;
    sim_status st = read_problem(grid, gas, bc, h->pb, nullptr);
    int lay[6];
    if (st == SIM_OK && (bc->tol != 0.0 || !strip_layout(h->pb.nx, n_strips, 0, lay))) st = SIM_EINVAL;
    if (st != SIM_OK) {
        sim_strips_destroy(h);
        return st;
    }
    Template t;
    make_template(h->pb, t);
    for (int k = 0; k < n_strips; k++) {
        strip_layout(h->pb.nx, n_strips, k, lay);
        sim_t s = new (std::nothrow) sim_s;
        if (!s) {
            sim_strips_destroy(h);
            return SIM_ENOMEM;
        }
        s->pb = h->pb;
        s->stream = h->stream;
        s->own0 = lay[0];
        s->own_stop = k == n_strips - 1 ? 0 : lay[1];
        st = build_handle(s, t, lay[2], lay[3]);
        if (st != SIM_OK) {
            sim_destroy(s);
            sim_strips_destroy(h);
            return st;
        }
        h->strip.push_back(s);
        h->own0.push_back(lay[0]);
        h->own1.push_back(lay[1]);
    }
    // the halo copies of each level: at the boundary X between strips k and
    // k + 1, the columns [X - halo, X) of strip k go to strip k + 1 and the
    // columns [X, X + halo) of strip k + 1 go to strip k, every row of the
    // extended grid, every field of the arithmetic's levels
    const int rows = h->pb.ny + 2 * G + 1;
    std::vector<HaloCopy> copies;
    for (int l = 0; l < 3; l++) {
        for (int k = 0; k + 1 < n_strips; k++) {
            sim_t a = h->strip[k], b = h->strip[k + 1];
            const int X = h->own1[k];
            void *pa[12], *pb[12];
            int ba[12], bb[12];
            const int n = level_arrays(a, l, pa, ba);
            level_arrays(b, l, pb, bb);
            for (int f = 0; f < n; f++) {
                const int e = ba[f];
                auto at = [&](void *base, int i) { return (unsigned *)((char *)base + (size_t)(i + G) * e); };
                const int wpitch_a = a->pitch * e / 4, wpitch_b = b->pitch * e / 4, words = kStripHalo * e / 4;
                copies.push_back(HaloCopy{at(pa[f], X - kStripHalo), at(pb[f], X - kStripHalo), wpitch_a, wpitch_b,
                                          words, rows});
                copies.push_back(HaloCopy{at(pb[f], X), at(pa[f], X), wpitch_b, wpitch_a, words, rows});
                h->max_words = std::max(h->max_words, words * rows);
            }
        }
        if (l == 0) h->n_copies = (int)copies.size();
    }
    const size_t stage = (size_t)(h->pb.nx + 1) * (h->pb.ny + 1);
    if ((!copies.empty() && cudaMalloc(&h->d_copies, copies.size() * sizeof(HaloCopy)) != cudaSuccess) ||
        cudaMalloc(&h->d_stage, stage * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->h_res, 4 * sizeof(unsigned long long) * n_strips) != cudaSuccess) {
        sim_strips_destroy(h);
        return SIM_ENOMEM;
    }
    if (!copies.empty() && cudaMemcpy(h->d_copies, copies.data(), copies.size() * sizeof(HaloCopy),
                                      cudaMemcpyHostToDevice) != cudaSuccess) {
        sim_strips_destroy(h);
        return SIM_ECUDA;
    }
    *out = h;
    return SIM_OK;
}

extern "C" sim_status sim_strips_step(sim_strips_t h, int n_steps, int scheme)
{
    if (!h) return SIM_EINVAL;
    if (n_steps < 0 || (scheme & ~3)) return sfail(h, SIM_EINVAL, "bad n_steps %d or scheme %d", n_steps, scheme);
    const bool implicit = scheme & SIM_IMPLICIT, tvd = scheme & SIM_TVD;
    for (int step = 0; step < n_steps; step++) {
        sim_strips_s::Graph &g = h->graphs[h->cur][scheme];
        if (!g.exec) {
            if (!h->cap_stream)
                SCUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            SCUDA_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
            g.result = enqueue_strips_step(h, h->cur, implicit, tvd, h->cap_stream);
            SCUDA_TRY(h, cudaStreamEndCapture(h->cap_stream, &graph));
            cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                g.exec = nullptr;
                return sfail(h, SIM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
            }
        }
        SCUDA_TRY(h, cudaGraphLaunch(g.exec, h->stream));
        h->cur = g.result;
        for (sim_t s : h->strip) {
            s->cur = h->cur;
            s->last_iters = h->pb.iters;
        }
    }
    SCUDA_TRY(h, cudaGetLastError());
    return SIM_OK;
}

extern "C" sim_status sim_strips_fields(sim_strips_t h, int field, double *host_dst, size_t n)
{
    if (!h) return SIM_EINVAL;
    if (field < 0 || field > 5 || !host_dst) return sfail(h, SIM_EINVAL, "bad field %d or null destination", field);
    const size_t need = field_count(h->pb, field);
    if (n != need) return sfail(h, SIM_EINVAL, "field %d has %zu elements, got %zu", field, need, n);
    const int ns = (int)h->strip.size();
    for (int k = 0; k < ns; k++) {
        sim_t s = h->strip[k];
        const int i1 = k == ns - 1 ? h->pb.nx + 1 : h->own1[k];
        if (s->df)
            launch_join(alloc_of(s->dfm.lv[h->cur], s->shift), alloc_of(s->lv[h->cur], s->shift), s->nelem, h->stream);
        if (s->mixed)
            launch_widen_mixed(s->geo, s->lv[h->cur], s->mx.lv[h->cur], s->sides.kind[SIDE_E] == BC_OUTFLOW,
                               h->own0[k], i1, h->stream);
        launch_gather_cols(s->geo, field, s->lv[h->cur], h->d_stage, h->own0[k], i1, h->stream);
    }
    SCUDA_TRY(h, cudaGetLastError());
    SCUDA_TRY(h, cudaMemcpyAsync(host_dst, h->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SCUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SIM_OK;
}

extern "C" sim_status sim_strips_residuals(sim_strips_t h, double out[4])
{
    if (!h || !out) return SIM_EINVAL;
    const int ns = (int)h->strip.size();
    for (int k = 0; k < ns; k++)
        SCUDA_TRY(h, cudaMemcpyAsync(h->h_res + 4 * k, h->strip[k]->work.res, 4 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, h->stream));
    SCUDA_TRY(h, cudaStreamSynchronize(h->stream));
    // the maxima over the strips: the same ordered keys the kernels reduce
    unsigned long long m[4] = {0, 0, 0, 0};
    for (int k = 0; k < ns; k++)
        for (int q = 0; q < 4; q++) m[q] = std::max(m[q], h->h_res[4 * k + q]);
    if (!read_residuals(m, out)) return sfail(h, SIM_EDIVERGED, "non-finite residual");
    return SIM_OK;
}

extern "C" const char *sim_strips_last_error(sim_strips_t h)
{
    return h ? h->err : "null handle";
}

extern "C" void sim_strips_destroy(sim_strips_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &row : h->graphs)
        for (auto &g : row)
            if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->d_copies);
    cudaFree(h->d_stage);
    if (h->h_res) cudaFreeHost(h->h_res);
    for (sim_t s : h->strip) sim_destroy(s);
    delete h;
}
