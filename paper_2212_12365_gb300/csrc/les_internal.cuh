// Internal definitions of libles.so shared by the kernels and the host runtime.
//
// Device layout (per jet): structure of arrays, field-major; inside a field
// the point (i,j,k) sits at (k*nj + j)*pitch + i with the row pitch padded to
// 128 bytes, so that every row starts on a 128-byte line and a warp reading 32
// consecutive i touches whole lines.  Padding columns are never read.
#pragma once

#include <cstdint>
#include <cuda.h> // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "les.h"

namespace les {

constexpr int NF = 5;         // conserved variables
// Static per-point grid fields (computed once in FP64, stored in the state
// precision): the nine metric cofactors J^-1 d xi^a / d x_c at [3a + c],
// J^-1, (Cs Delta)^2, J, and per axis a: half the J^-1 average of the
// interface to the +a neighbour, the reciprocal of that average (not halved),
// and |row a| = sqrt(sum_c m_ac^2).
constexpr int NMET = 21;      // fields of every precision
constexpr int MET_A0 = 21;    // FP64 only: 27 interface tables, see below
constexpr int MET_K0 = 48;    // FP64 only: 9 interface contractions, see below
constexpr int NMET64 = 57;
constexpr int MET_JINV = 9;
constexpr int MET_CSD2 = 10;
constexpr int MET_J = 11;
constexpr int MET_JB = 12;    // + a
constexpr int MET_RJB = 15;   // + a
constexpr int MET_NORM = 18;  // + a
// FP64 only, per axis a at [MET_A0 + 9a + 3b + c]: the interface (to the +a
// neighbour) average of the cofactor J^-1 d xi^b / d x_c divided by the
// interface J^-1, times 1/2 for b != a: the chain-rule weights of the compact
// viscous flux applied to the normal difference (b == a) and to the SUM of
// the two points' central differences (b != a).
// FP64 only, per axis a at [MET_K0 + 3a + b]: K_b = sum_c A_ac A_bc (same
// tables), so that the flux-direction contraction of a gradient,
// sum_c A_ac d phi/d x_c, is sum_b K_b D_b.
// Per-point stage fields: primitives, Sutherland viscosity, lambda-bar,
// the unscaled conserved vector W0..W3 (= rho is P_RHO) and rho H = e + p,
// and the inviscid point fluxes F_a (5 each) at P_F0 + 5a + f.
constexpr int NPRIM = 29;
enum {
    P_RHO = 0, P_U, P_V, P_W, P_P, P_T, P_MU, P_LXI, P_LETA, P_LZETA,
    P_RU, P_RV, P_RW, P_RH, P_F0
};
// Per-point derivative fields: d(u,v,w,T)/d(xi,eta,zeta) at [3*phi + axis],
// mu_sgs, mu/Re + mu_sgs, the total conductivity, and the pressure sensor
// per axis.
constexpr int NGRAD = 18;
constexpr int G_MUSGS = 12;
constexpr int G_MUEFF = 13;
constexpr int G_KAP = 14;
constexpr int G_NU = 15;      // + a
constexpr int NHF = 15;       // interface fluxes H_a at [5a + f], interface L + e_a/2

constexpr int BLOCK = 256;    // threads per block of the point / face kernels
constexpr int DBG_RHS = 100;  // debug export codes beside the LES_FIELD_* values
constexpr int DBG_MET0 = 200;

// Geometry and parameters of one jet, as seen by the kernels.
template <typename real>
struct JetDev {
    int n[3];          // ni, nj, nk
    int pitch;         // padded row length (elements)
    long long fs;      // field stride (elements)
    int per[3];
    int bc[6];
    // state registers of the 5-stage scheme: q[0] = Q(0) (and the step result),
    // q[1], q[2] ping-pong stage registers
    real *q[3];
    const real *met;   // NMET fields
    const double *jinv64; // J^-1 in FP64 (conversions of the state, Qhat sums)
    real *prim;        // NPRIM fields (scratch, rebuilt every stage)
    real *grad;        // NGRAD fields (scratch)
    real *hflux;       // NHF fields (scratch): interface fluxes
    real *rhs;         // NF fields (residual for diagnostics / debug)
    const double *inflow_ut; // nj*nk: inflow profile u~(r) of the i = 0 face points (host tanh)
    // flow parameters (jet units)
    double gamma, Pr, Pr_sgs, Re, mach, TR, theta, noise_amp, k2, k4, suth_S;
    double gm1, suth1; // gamma - 1, 1 + suth_S
    double inv_Re;     // 1/Re (0 for an inviscid run)
    double kap_mol;    // mu -> conductivity: 1/(Re Pr (gamma-1))
    double kap_sgs;    // mu_sgs -> conductivity: 1/(Pr_sgs (gamma-1))
    double bc_g1, bc_rg, bc_cinf; // 1/(gamma-1), 1/gamma, ambient sound speed (1/TR)^1/2
    unsigned long long seed;
    long long npts_pad; // nk*nj*pitch
    // first out-of-range index met by a kernel of a LES_BOUNDS_CHECK build
    // (see bounds_ok); unused otherwise
    unsigned long long *oob;
};

// Block map of a batched launch: virtual block vb belongs to jet j when
// start[j] <= vb < start[j+1].
struct BlockMap {
    const int *start;  // njets + 1 entries (device)
    int njets;
    int total;
};

__device__ __forceinline__ int find_jet(const BlockMap &bm, int vb)
{
    int lo = 0, hi = bm.njets; // start[lo] <= vb < start[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(bm.start + mid) <= vb) lo = mid; else hi = mid;
    }
    return lo;
}

// Index-bounds checking of a debug build (compiled with -DLES_BOUNDS_CHECK,
// the stand-in for a memory checker): an index outside [0, n) is recorded
// in *oob as (site << 48) | (index & 2^48-1), first violation wins, and the
// access is redirected to index 0 instead of faulting.  In a normal build
// the checks compile to nothing.  Sites: 1 point index (lidx), 2-4 global
// offsets of the fused stage (state / static record / update), 5-7 its
// shared-memory slots (point ring / plane tables / eta-flux rows).
#if defined(LES_BOUNDS_CHECK) && defined(__CUDA_ARCH__)
__device__ __forceinline__ void bounds_record(unsigned long long *oob, int site, unsigned long long v)
{
    if (oob) atomicCAS(oob, 0ull, ((unsigned long long)site << 48) | (v & 0xFFFFFFFFFFFFull));
}
__device__ __forceinline__ long long bounds_ok(unsigned long long *oob, int site, long long idx, long long n)
{
    if (idx >= 0 && idx < n) return idx;
    bounds_record(oob, site, (unsigned long long)idx);
    return 0;
}
#define LES_BOUNDS(oob, site, idx, n) bounds_ok((oob), (site), (long long)(idx), (long long)(n))
#else
#define LES_BOUNDS(oob, site, idx, n) (idx)
#endif

template <typename real>
__host__ __device__ __forceinline__ long long lidx(const JetDev<real> &J, int i, int j, int k)
{
#if defined(LES_BOUNDS_CHECK) && defined(__CUDA_ARCH__)
    // a component out of its axis (recorded as 16-bit i, j, k) could still
    // land inside the array, so the components are checked
    if (i < 0 || i >= J.n[0] || j < 0 || j >= J.n[1] || k < 0 || k >= J.n[2]) {
        bounds_record(J.oob, 1, ((unsigned long long)(k & 0xFFFF) << 32) | ((unsigned long long)(j & 0xFFFF) << 16) |
                                    (unsigned long long)(i & 0xFFFF));
        return 0;
    }
#endif
    return ((long long)k * J.n[1] + j) * J.pitch + i;
}

// Scale of the stored state Qhat = s Q at a point: J^-1, or 1 on the
// degenerate axis of a polar mesh (centerline face), where J^-1 = 0 and the
// state is kept unscaled (Sec. "Centerline Boundary Condition").
__host__ __device__ __forceinline__ double state_scale(double jinv) { return jinv > 0.0 ? jinv : 1.0; }

// Scale of the state as stored by a handle of storage type `real`.  FP64
// handles store Qhat = J^-1 Q, the variable the Runge-Kutta scheme advances.
// FP32 handles store the unscaled Q and advance it as Q(l) = Q(0) - alpha_l
// dt J RHS, the same update multiplied by J: a uniform state is then stored
// exactly alike at every point, whereas FP32 rounding of J^-1 Q on a
// stretched grid seeds a point-to-point pressure noise that drives the
// transverse momenta.
template <typename real> __host__ __device__ __forceinline__ double stored_scale(double jinv)
{
    if constexpr (sizeof(real) == sizeof(float)) return 1.0;
    else return state_scale(jinv);
}

__host__ __device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

#ifdef __CUDACC__
// Unit stencil of a second-order first derivative along one axis with
// Delta xi = 1: central, or one-sided 3-point at the ends of a non-periodic
// axis.  off[] are index offsets, wgt[] the weights.
struct Stencil {
    int n;
    int off[3];
    double wgt[3];
};

__device__ __forceinline__ Stencil deriv_stencil(int q, int n, int periodic)
{
    Stencil s;
    if (periodic || (q > 0 && q < n - 1)) {
        s.n = 2;
        s.off[0] = -1; s.wgt[0] = -0.5;
        s.off[1] = 1;  s.wgt[1] = 0.5;
        s.off[2] = 0;  s.wgt[2] = 0.0;
    } else if (q == 0) {
        s.n = 3;
        s.off[0] = 0; s.wgt[0] = -1.5;
        s.off[1] = 1; s.wgt[1] = 2.0;
        s.off[2] = 2; s.wgt[2] = -0.5;
    } else {
        s.n = 3;
        s.off[0] = 0;  s.wgt[0] = 1.5;
        s.off[1] = -1; s.wgt[1] = -2.0;
        s.off[2] = -2; s.wgt[2] = 0.5;
    }
    return s;
}

// Point (i,j,k) of padded linear index lp; false for padding columns.

template <typename real>
__device__ __forceinline__ bool point_of(const JetDev<real> &J, long long lp, int q[3])
{
    int i = (int)(lp % J.pitch);
    long long r = lp / J.pitch;
    q[0] = i;
    q[1] = (int)(r % J.n[1]);
    q[2] = (int)(r / J.n[1]);
    return i < J.n[0] && q[2] < J.n[2];
}

template <typename real>
__device__ __forceinline__ bool is_end(const JetDev<real> &J, int a, int qa)
{
    return !J.per[a] && (qa == 0 || qa == J.n[a] - 1);
}

template <typename real>
__device__ __forceinline__ bool interior(const JetDev<real> &J, const int q[3])
{
    return !(is_end(J, 0, q[0]) || is_end(J, 1, q[1]) || is_end(J, 2, q[2]));
}

#endif

// Flow constants of one jet in FP32 for the fused stage kernel.
struct FusedParams {
    float gam, gm1, hgam;   // gamma, gamma - 1, gamma / (gamma - 1)
    float k2, k4;           // Turkel-Vatsa constants
    float inv_Re, kap_mol, kap_sgs;
    float suth1, suthS;     // Sutherland: mu = T^1.5 suth1 / (T + suthS)
    float cs2;              // Smagorinsky C_s^2 (separable form: (C_s Delta)^2 = cs2 (h_x h_y h_z)^(2/3))
    float pinf;             // ambient pressure 1/gamma: subtracted from p in the pressure flux terms
};

// Work-list entry of one jet for the fused stage kernel: items
// [item0, item0 + nbx*nby*nkc) are its (tile x, tile y, k-chunk) triples.  In
// the balanced form (kc == 0) the items are its tile-planes, nkc = the number
// of planes per column, and every CTA takes one contiguous range of them.
struct FusedJet {
    int item0;             // first work item of the jet
    int tile0;             // first tile of the jet (balanced form)
    int nbx, nby, nkc;
    int kc;                 // planes per k-chunk (0: balanced form)
    int njp;                // row pairs per column of the paired static records, (nj + 1) / 2
    FusedParams fp;
    // separable form (Cartesian-product grid): per axis a, for each index,
    // (h, 1/h, h^(2/3), 0) with h the derivative of coordinate a along axis a
    const float4 *h1[3];
    // general form: the static fields of the two points of each row pair
    // (rows 2p, 2p+1) of a column, interleaved point by point in five
    // float4: (m0 m1) (m2 m3) (m4 m5) (m6 m7) (m8, J^-1), m = the metric
    // cofactors; float4 number q of (i, pair p, k) at
    // ((k * njp + p) * 5 + q) * pitch + i, so that consecutive columns are
    // consecutive in memory for every q
    const float4 *mp;
    // jets with no periodic i or j axis: tensor maps of the three state
    // registers for the TMA staging of the next plane (null: plain loads)
    const CUtensorMap *tmap;
};

// TMA staging box of the fused stage: 5 fields x 1 plane x (TY + 4) rows x
// 40 columns (the tile's 34 columns plus up to 3 for aligning the start
// column down to a multiple of 4, i.e. 16 bytes).
constexpr int TMA_BOX_X = 40;
constexpr int tma_box_rows(int ty) { return ty + 4; }

// Error text of the handle-free entry points (les_last_error(NULL)).
void set_call_error(const char *msg);

template <int TY> int fused_prepare();
// resident CTAs per SM of the fused stage for tile height ty (general or
// separable form), from the occupancy calculator; 1 if it cannot tell
int fused_ctas_per_sm(int ty, int separable);
// One launch of the fused stage.  jets / fj: the device tables of the njets
// jets; for a single jet (njets == 1) j1 / f1 are host copies of its two
// entries, passed by value as kernel parameters, so that the kernel reads the
// jet's constants from the parameter bank (null otherwise).
template <int TY>
void launch_fused(const JetDev<float> *jets, const FusedJet *fj, int njets, int total_items, int total_tiles,
                  int grid, int src, int dst, int stage, const double *dt, int rhs_only, int separable, int balanced,
                  int wait_limit, const JetDev<float> *j1, const FusedJet *f1, cudaStream_t st);

// General FP32 form: the paired static records (see FusedJet::mp) from the
// FP32 static fields; mp holds nk * ((nj + 1) / 2) * 5 * pitch float4.
void launch_pack_pairs(const float *met, long long fs, int pitch, int nj, int nk, float4 *mp, cudaStream_t st);
// Separable form: 1-D spacings of a Cartesian-product grid from device
// coordinates (FP64 derivative stencils of the metric computation).
void launch_sep_metrics(const double *x, const double *y, const double *z, const int n[3], const int per[3],
                        const double shift[9], float4 *h1x, float4 *h1y, float4 *h1z, cudaStream_t st);

// Kernel launchers (les_kernels.cu, les_stage.cu), all asynchronous on `st`.
template <typename real> struct Launch {
    static void metrics(const double *x, const double *y, const double *z, int ni, int nj, int nk,
                        const int per[3], const double shift[9], double *met64, long long fs64,
                        int pitch, double Cs, cudaStream_t st);
    static void convert_metrics(const double *met64, long long fs64, real *met, long long fs,
                                long long npad, cudaStream_t st);
    static void static_fields(double *met64, long long fs64, int pitch, const int n[3],
                              const int per[3], int iface_tables, cudaStream_t st);
    static void point(const JetDev<real> *jets, BlockMap bm, int src, int grid, cudaStream_t st);
    static void grads(const JetDev<real> *jets, BlockMap bm, int grid, cudaStream_t st);
    static void iface(const JetDev<real> *jets, BlockMap bm, int grid, cudaStream_t st);
    static void update(const JetDev<real> *jets, BlockMap bm, int dst, int stage,
                       const double *dt, int rhs_only, int grid, cudaStream_t st);
    static void bc(const JetDev<real> *jets, BlockMap bm, int axis, int dst,
                   const long long *level, int grid, cudaStream_t st);
    static void set_state(const JetDev<real> *jets, int jet, const double *in, int kind,
                          long long npad, cudaStream_t st);
    static void get_state(const JetDev<real> *jets, int jet, double *out, int kind,
                          long long npad, cudaStream_t st);
    static void dt_max(const JetDev<real> *jets, BlockMap bm, unsigned long long *maxbits,
                       int grid, cudaStream_t st);
    static void diag_partials(const JetDev<real> *jets, int jet, double *partials, int nblocks,
                              cudaStream_t st);
    // field: LES_FIELD_* (not METRICS), DBG_RHS (5 fields) or DBG_MET0 + t (t < 10)
    static void debug_field(const JetDev<real> *jets, int jet, int field, double *out,
                            long long npad, cudaStream_t st);
    static void probe(const JetDev<real> *jets, const int *cell, const double *wts, int npts,
                      int every, const long long *level, const long long *base, real *out,
                      int capacity, cudaStream_t st);
};

// Centerline faces (j- face of type LES_BC_CENTERLINE) of jets [0, njets):
// the conserved variables of every axis point are the azimuthal mean of the
// adjacent ring j = 1.
template <typename real>
void launch_centerline(const JetDev<real> *jets, int njets, int max_ni, int dst, cudaStream_t st);

void launch_diag_final(const double *partials, int nblocks, double *out, cudaStream_t st);
void launch_step_advance(long long *level, cudaStream_t st);

} // namespace les
