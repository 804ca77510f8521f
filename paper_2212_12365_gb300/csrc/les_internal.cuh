// Internal definitions of libles.so shared by the kernels and the host runtime.
//
// Device layout (per jet): structure of arrays, field-major; inside a field
// the point (i,j,k) sits at (k*nj + j)*pitch + i with the row pitch padded to
// 128 bytes, so that every row starts on a 128-byte line and a warp reading 32
// consecutive i touches whole lines.  Padding columns are never read.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "les.h"

namespace les {

constexpr int NF = 5;         // conserved variables
constexpr int NMET = 11;      // J^-1 xi_x .. J^-1 zeta_z (9), J^-1, (Cs Delta)^2
constexpr int MET_JINV = 9;
constexpr int MET_CSD2 = 10;
constexpr int NPRIM = 10;     // rho u v w p T mu lbar_xi lbar_eta lbar_zeta
enum { P_RHO = 0, P_U, P_V, P_W, P_P, P_T, P_MU, P_LXI, P_LETA, P_LZETA };
constexpr int NGRAD = 13;     // d(u,v,w,T)/d(xi,eta,zeta) as [phi*3 + axis], mu_sgs
constexpr int G_MUSGS = 12;

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
    const double *jinv64; // J^-1 in FP64 (conversions of the state)
    real *prim;        // NPRIM fields (scratch, rebuilt every stage)
    real *grad;        // NGRAD fields (scratch)
    real *rhs;         // NF fields (residual for diagnostics / debug)
    const double *inflow_r; // nj*nk: radius sqrt(y^2+z^2) of the i = 0 face points
    // flow parameters (jet units)
    double gamma, Pr, Pr_sgs, Re, mach, TR, theta, noise_amp, k2, k4, suth_S;
    unsigned long long seed;
    long long npts_pad; // nk*nj*pitch
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

template <typename real>
__host__ __device__ __forceinline__ long long lidx(const JetDev<real> &J, int i, int j, int k)
{
    return ((long long)k * J.n[1] + j) * J.pitch + i;
}

__host__ __device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// Kernel launchers (les_kernels.cu), all asynchronous on `st`.
template <typename real> struct Launch {
    static void metrics(const double *x, const double *y, const double *z, int ni, int nj, int nk,
                        const int per[3], const double shift[9], double *met64, long long fs64,
                        int pitch, double Cs, cudaStream_t st);
    static void convert_metrics(const double *met64, long long fs64, real *met, long long fs,
                                long long npad, cudaStream_t st);
    static void prims(const JetDev<real> *jets, BlockMap bm, int src, int grid, cudaStream_t st);
    static void grads(const JetDev<real> *jets, BlockMap bm, int grid, cudaStream_t st);
    static void flux(const JetDev<real> *jets, BlockMap bm, int src, int dst, int stage,
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

void launch_diag_final(const double *partials, int nblocks, double *out, cudaStream_t st);
void launch_step_advance(long long *level, cudaStream_t st);

} // namespace les
