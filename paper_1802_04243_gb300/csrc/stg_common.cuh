// stg_common.cuh -- data layout shared by the host driver and the sweep
// kernels of the SIMPLE-TS time step (arXiv:1802.04243, Section 3).
//
// Every field lives in one device array of (ny + 5) rows x pitch doubles.
// Element (i, j) of any field -- cell centre, u face (x^f_i, y^v_j) or v face
// (x^v_i, y^f_j) -- sits at IX(i, j) = (j + G) * pitch + (i + G), with two
// ghost layers (G = 2) on every side.  Cells use i in [-2, nx+1], u faces
// i in [-2, nx+2], v faces j in [-2, ny+2].
#pragma once

#include <cstddef>
#include <cuda_runtime.h>
#include <cstdint>

#include "df64.cuh"

namespace stg {

using dfl::df64;

constexpr int G = 2;

// Per-node geometry flags, one uint16 per extended grid position (i, j).
enum : uint32_t {
    F_FLUID = 1u << 0,    // cell (i,j) is fluid (an unknown of T and p)
    F_WALL = 1u << 1,     // cell (i,j) is a wall ghost or obstacle cell
    F_UACT = 1u << 2,     // u face (i,j) lies between two fluid cells
    F_UWALL = 1u << 3,    // u face (i,j) lies inside a wall or obstacle
    F_VACT = 1u << 4,     // v face (i,j) lies between two fluid cells
    F_VWALL = 1u << 5,    // v face (i,j) lies inside a wall or obstacle
    F_TCX = 1u << 6,      // cells i-2..i+1 of row j are fluid (TVD on x face i)
    F_TCY = 1u << 7,      // cells j-2..j+1 of column i are fluid (TVD on y face j)
    F_TUX = 1u << 8,      // u faces i-2..i+1 of row j are unknowns
    F_TUY = 1u << 9,      // u faces j-2..j+1 of column i are unknowns
    F_TVX = 1u << 10,     // v faces i-2..i+1 of row j are unknowns
    F_TVY = 1u << 11,     // v faces j-2..j+1 of column i are unknowns
    F_INTERIOR = 1u << 12, // no wall within two cells of any position of the aligned 32-wide
                           // row segment holding (i,j): cells [32k-2, 32k+33] x [j-2, j+2] are fluid
};

// Per-index grid factors, each array indexed by i + G (x) or j + G (y) over
// the extended range [-2, n + 2].
template <typename R>
struct AxisT {
    const R *d;      // cell size
    const R *rd;     // 1 / d
    const R *wlo;    // d_i / (d_{i-1} + d_i): weight of index i-1 at face i
    const R *whi;    // d_{i-1} / (d_{i-1} + d_i): weight of index i at face i
    const R *rc;     // 1 / (0.5 (d_{i-1} + d_i)): inverse centre distance across face i
    // Weights of the derivative across cell i of a quantity interpolated to
    // faces i and i+1 and averaged over two rows: with a pair sum S(k) of the
    // two rows' values at index k, (f_{i+1} - f_i) / d_i equals
    // qlo * -S(i-1) + qmid * S(i) + qhi * S(i+1).
    const R *qlo;    // wlo_i / (2 d_i)
    const R *qmid;   // (wlo_{i+1} - whi_i) / (2 d_i)
    const R *qhi;    // whi_{i+1} / (2 d_i)
    const R *dc;     // 0.5 (d_{i-1} + d_i): centre distance across face i
    const R *wlo2;   // 2 wlo (exact): the TVD face corrections take twice the weight
    const R *whi2;   // 2 whi
    const R *hd;     // 0.5 d_i (exact)
    const R *ddt;    // d_i / (2 dt): the transient factor of the momentum control volumes
    const R *ct2d;   // 2 C^T1_f d_i: twice the conductance factor of a face of length d_i (Eq. pl32)
    const R *dt1;    // d_i / dt: with the other axis's d, a cell's volume per unit time
};

// Number of per-index arrays of an axis table, stored one after another.
constexpr int kAxisTables = 15;

// The arrays of an axis table of m entries per array starting at t.
template <typename R>
inline AxisT<R> axis_view(const R *t, int m)
{
    return AxisT<R>{t,         t + m,     t + 2 * m, t + 3 * m, t + 4 * m,  t + 5 * m,  t + 6 * m,
                    t + 7 * m, t + 8 * m, t + 9 * m, t + 10 * m, t + 11 * m, t + 12 * m, t + 13 * m, t + 14 * m};
}

template <typename R>
struct GeoT {
    int nx, ny;
    int pitch;
    const uint16_t *flag;
    AxisT<R> x, y;
};

template <typename R>
struct CoefT {
    R A, B, CT1f, CT2f, CT3f, omega, dt, gx, gy;
    R hrdt;               // 0.5 / dt
    R zeta, tau;          // slip / jump coefficients (Eqs. pl38, pl39), divided by rho_local at use; 0 = off
    R B23;                // 2/3 B, the factor of the normal-stress cross terms of Eqs. pl14, pl16
};

// One state level: u, v at faces; p, T, rho, Gamma at cell centres.
template <typename R>
struct LevelT {
    R *u, *v, *p, *T, *rho, *gam;
};

// Scratch of one loop-2 iteration (all extended-indexed).  The arrays are
// carved one after another in this order; kWorkArrays counts them.
template <typename R>
struct WorkT {
    R *ru_dy, *rv_dx;              // face densities (Eqs. pl10, pl11) times the face area: rho^u dy, rho^v dx
                                   // (FP64: the assembly replaces them by a^px = rho^u dy d^u and
                                   // a^py = rho^v dx d^v, the pressure kernel's coefficients, Eq. pl24)
    R *Fx, *Fy;                    // mass fluxes F^x = rho^u u dy, F^y = rho^v v dx (Eqs. pl8, pl9)
    R *DTx, *DTy;                  // T conductances of x and y faces, C^T1_f Gamma_harm dy / dx_c (Eqs. pl32, pl33)
    R *Bgc;                        // B Gamma at the corner (x^f_i, y^f_j), bilinear in the four cells
    R *Bgx, *Bgy;                  // B Gamma dy/dx and B Gamma dx/dy of cell (i,j): normal-stress conductances
    R *Fbu, *Fbv;                  // mass fluxes through the centre of cell (i,j) between the u (v) control
                                   // volumes: rho 0.5 (u_i + u_{i+1}) dy and rho 0.5 (v_j + v_{j+1}) dx
    R *Su, *Sv;                    // u_i + u_{i+1} and v_j + v_{j+1} of cell (i,j), the pair sums of the
                                   // energy source's dv/dx, du/dy (stored by the FP64 and DF64 sweeps)
    R *uhat, *du, *vhat, *dv;      // pseudo velocities and d (Eqs. pl14, pl20, pl21)
    // TVD limiters of one level, one evaluation per face (Eqs. pl15_1, pl15_2;
    // 0 where the face's stencil is not all unknowns): T on the x and y faces;
    // u on the x face of its control volume (at the centre of cell i-1) and
    // on the y face below node (i,j) for flow up (U) and down (D); v likewise
    R *psTx, *psTy, *psUx, *psUyU, *psUyD, *psVy, *psVxU, *psVxD;
    R *uexp, *vexp, *Texp;         // explicit convective terms (Eqs. pl15_11, pl31_1)
    R *bpx, *bpy;                  // FP64: rho^u dy u^ and rho^v dx v^ of the faces, the pressure
                                   // equation's source fluxes (Eq. pl24), stored by the assembly
    R *Bgcu, *Bgcv;                // FP64: B Gamma at the corner (i,j) times dc_x(i)/dc_y(j) and times
                                   // dc_y(j)/dc_x(i): the diffusive conductances of the u control
                                   // volumes' y faces and of the v control volumes' x faces
};

constexpr int kWorkArrays = 32;
// Arrays of one pool: three levels of six fields, then the scratch.
constexpr int kPoolArrays = 3 * 6 + kWorkArrays;

using Axis = AxisT<double>;
using Geo = GeoT<double>;
using Coef = CoefT<double>;
using Level = LevelT<double>;

struct Work : WorkT<double> {
    unsigned long long *res;       // 4 residual maxima as ordered bit patterns
};

// FP32 side of the mixed-precision sweep: FP32 grid factors and
// coefficients, FP32 levels (written from the FP64 ones whenever a level is
// set; during the sweep they carry u, v, T and Gamma, whose FP64 values are
// filled when the state is read) and FP32 iteration scratch.
struct Mixed {
    GeoT<float> g;
    CoefT<float> k;
    LevelT<float> lv[3];
    WorkT<float> w;
};

// Double-float side of the DF64 sweep: grid factors, coefficients, the three
// working state levels and the iteration scratch, all double-float.  The FP64
// levels are filled from them only when the state is read out.
struct DoubleFloat {
    GeoT<df64> g;
    CoefT<df64> k;
    LevelT<df64> lv[3];
    WorkT<df64> w;
};

// Arithmetic of the equation kernels.
enum { PREC_FP64 = 0, PREC_MIXED = 1, PREC_DF64 = 2 };

// One problem of a tile list, as the equation kernels see it (device resident).
struct Inst {
    Geo g;
    Coef k;
    GeoT<float> g32;
    CoefT<float> k32;
    GeoT<df64> gdf;
    CoefT<df64> kdf;
    Level lv[3];
    LevelT<float> lv32[3];
    LevelT<df64> lvdf[3];
    Work w;
    WorkT<float> w32;
    WorkT<df64> wdf;
    int east_outflow;
    int tiles_x;          // tiles along x for the batch's tile shape
    int tile0;            // index of this problem's first tile in the batch
    // One strip of a problem decomposed along x (all 0 for a whole problem):
    // the tiles start at column x0; positions of columns >= x_stop (when
    // x_stop > 0) are skipped; the residual maxima take only the columns in
    // [own0, own_stop) (own_stop 0: no upper limit).
    int x0, x_stop, own0, own_stop;
};

// Work distribution of the equation kernels: tiles of tx x ty threads
// (tx * ty <= 256) over every problem of the list, walked by `grid` CTAs
// (the assembly kernel by `grid_asm` CTAs when that is positive).
struct BatchPlan {
    const Inst *inst;
    const int *tile_inst; // problem of each tile
    int n_inst, n_tiles;
    int tx, ty, grid;
    Inst one;             // copy of inst[0], read from the launch parameters when n_inst == 1
    int grid_asm;         // CTAs of the assembly kernel; 0: grid
};

// Boundary description used by the ghost refresh.
struct Sides {
    int kind[4];          // W, E, S, N
    int col0, col1;       // columns [col0, col1) the S/N refresh covers; col1 = 0: [-2, nx + 2]
};

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
// BC_INTERFACE: the side of an x-strip that faces another strip (its halo is
// copied from the neighbour, no ghost rule applies)
enum { BC_WALL = 0, BC_SYMMETRY = 1, BC_INFLOW = 2, BC_OUTFLOW = 3, BC_INTERFACE = 4 };

// Launch wrappers (sweep_kernels.cu; the equation kernels' own launchers in
// phase_kernels.cuh).  All are asynchronous on `stream`.
//
// Equation kernels: one launch per phase over a tile list (one problem or a
// batch).  `prec` (PREC_*) selects the arithmetic: FP64; the FP32 assembly
// of the mixed-precision path; double-float.  Levels are indices into
// Inst::lv / lv32 / lvdf.
// The face kernel also resets the residual words of every problem of the
// list (its first CTA), since it opens every loop-2 iteration.
// limiters: also store the TVD limiters of the level (tvd only; the kernels
// that read them are the implicit-TVD assembly and the explicit terms).
void launch_faces(const BatchPlan &bp, int prec, int level, bool tvd, bool limiters, void *stream);
void launch_explicit(const BatchPlan &bp, int prec, int prev, bool tvd, void *stream);
void launch_assemble(const BatchPlan &bp, int prec, int prev, int old, int nw, bool implicit, bool tvd,
                     void *stream);
void launch_pressure(const BatchPlan &bp, int prec, int prev, int old, int nw, void *stream);
void launch_velocity(const BatchPlan &bp, int prec, int old, int nw, void *stream);
// The same for one arithmetic (PREC_*), each compiled in a translation unit
// of its own (phase_kernels.cuh; lim: store the TVD limiters).
template <int PREC>
void launch_faces_of(const BatchPlan &bp, int level, bool tvd, int lim, void *stream);
template <int PREC>
void launch_explicit_of(const BatchPlan &bp, int prev, bool tvd, void *stream);
template <int PREC>
void launch_assemble_of(const BatchPlan &bp, int prev, int old, int nw, bool implicit, bool tvd, void *stream);
template <int PREC>
void launch_pressure_of(const BatchPlan &bp, int prev, int old, int nw, void *stream);
template <int PREC>
void launch_velocity_of(const BatchPlan &bp, int old, int nw, void *stream);
// The persistent step kernel of one arithmetic (k_step, phase_kernels.cuh).
template <int PREC>
void *step_kernel_for(bool implicit, bool tvd);

// Persistent step of a batch (persistent.cu): one cooperative kernel runs a
// list of phases over the tile list, a grid barrier between each two.
enum { PH_FACES = 0, PH_EXPLICIT = 1, PH_ASSEMBLE = 2, PH_PRESSURE = 3, PH_VELOCITY = 4 };
constexpr int kMaxPhases = 64;
struct PhaseList {
    int n;
    unsigned char kind[kMaxPhases];
    unsigned char a[kMaxPhases], b[kMaxPhases], c[kMaxPhases];   // the phase's level arguments
};
struct GridBarrier {
    unsigned count, gen, err, pad;   // err != 0: a barrier wait ran out of time
};
// CTAs of the persistent kernel that stay resident together (0 on error).
int persistent_ctas(int prec, bool implicit, bool tvd, int threads);
// Clears the barrier and launches one step (cooperative launch, `ctas` CTAs).
cudaError_t launch_step_persistent(const BatchPlan &bp, const PhaseList &ph, GridBarrier *bar, int prec, bool implicit,
                                   bool tvd, int ctas, void *stream);

// Ghost copies of outflow and symmetry sides.  after_velocity: the velocity
// kernel has already copied the outflow side, only symmetry sides remain.
void launch_ghosts(const Geo &g, const Sides &s, const Level &lv, bool after_velocity, void *stream);
void launch_ghosts_f32(const Mixed &m, const Sides &s, int level, bool after_velocity, void *stream);
void launch_ghosts_df(const DoubleFloat &d, const Sides &s, int level, bool after_velocity, void *stream);
int ghost_kernels(const Sides &s, bool after_velocity);

// State maintenance.  The _cols variants cover the columns [i0, i1) only.
void launch_derive(const Geo &g, const Coef &c, const Level &lv, void *stream);
void launch_derive_cols(const Geo &g, const Coef &c, const Level &lv, int i0, int i1, void *stream);
void launch_scatter(const Geo &g, int field, const double *src, const Level &lv, void *stream);
void launch_gather(const Geo &g, int field, const Level &lv, double *dst, void *stream);
void launch_gather_cols(const Geo &g, int field, const Level &lv, double *dst, int i0, int i1, void *stream);
// The FP64 u, v, T and Gamma of a mixed-precision level over columns
// [i0, i1), from their FP32 values where the sweep computes them, and the
// outflow ghost copies when the east side is an outflow: the mixed sweep keeps
// those four fields in FP32 only.
void launch_widen_mixed(const Geo &g, const Level &lv, const LevelT<float> &s32, bool east_outflow, int i0, int i1,
                        void *stream);

// Halo exchange of an x-decomposed problem: n copies of a block of `rows`
// rows x `words` 4-byte words between two arrays (row pitches in words),
// one launch for every copy of a loop-2 iteration.
struct HaloCopy {
    const unsigned *src;
    unsigned *dst;
    int spitch, dpitch;   // words per row
    int words, rows;      // block width in words, rows
};
void launch_halo_copies(const HaloCopy *copies, int n, int max_words, void *stream);
// The four state fields u, v, p, T as separate arrays in their logical shapes.
struct StatePtrs {
    double *f[4];
};
struct StateSrc {
    const double *f[4];
};
// All four fields in one launch.  The scatter reads them back to back from
// the staging array and derives rho and Gamma as launch_derive does; the
// gather writes four arrays (device memory, or page-locked host memory the
// device addresses); the staging copy reads four such arrays into the
// staging array and checks them as launch_validate_state does.
void launch_scatter_state(const Geo &g, const Coef &c, const double *stage, const Level &lv, void *stream);
void launch_gather_state(const Geo &g, const Level &lv, const StatePtrs &dst, void *stream);
void launch_stage_state(const StateSrc &src, size_t nu, size_t nv, size_t nc, double *stage, unsigned *bad,
                        void *stream);
// Sets *bad (|= 1) if a value of the staged u, v, p, T is not finite or p, T <= 0.
void launch_validate_state(const double *stage, size_t nu, size_t nv, size_t nc, unsigned *bad, void *stream);
void launch_shadow(const Geo &g, const Level &lv, const LevelT<float> &lv32, size_t nelem, void *stream);
// Whole-level conversions between FP64 and double-float (ghosts included).
void launch_split(const Level &lv, const LevelT<df64> &d, size_t nelem, void *stream);
void launch_join(const LevelT<df64> &d, const Level &lv, size_t nelem, void *stream);

// The FP64 reciprocal of the sweep (a series step from the FP32 reciprocal) and the
// IEEE quotient 1/x of each x[q], interleaved in out[2q], out[2q+1].
void launch_recip_check(const double *x, double *out, int n, void *stream);
// The FP64 square root of the sweep (Gamma = T^1/2: two Newton steps from the
// FP32 reciprocal square root) and the IEEE root of each x[q], interleaved.
void launch_sqrt_check(const double *x, double *out, int n, void *stream);

}  // namespace stg
