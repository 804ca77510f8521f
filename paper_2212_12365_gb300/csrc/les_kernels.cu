// CUDA kernels of libles.so (sm_103a).
//
// Grid setup (metrics and static fields), boundary conditions, state
// conversion, time step, diagnostics, debug export and probe kernels.  The
// Runge-Kutta stage kernels are in les_stage.cu.
//   k_bc : boundary faces of one axis (Sec. "Boundary Conditions"); launched
//          for y, then z, then x after every stage
// All per-point kernels are persistent grid-stride loops over a block map that
// spans one or many jets (batched form); the per-point arithmetic does not
// depend on the map, so a jet gives the same bits alone or in a batch.
#include <cmath>
#include <algorithm>
#include <cstdint>

#include "les_internal.cuh"

namespace les {

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int floordiv_i(int a, int n)
{
    int q = a / n;
    return (a % n != 0 && a < 0) ? q - 1 : q;
}

// ---------------------------------------------------------------------------
// Metric terms (FP64), Sec. "Transformation of Coordinates"
// ---------------------------------------------------------------------------

struct CoordGrid {
    const double *X[3];
    int n[3];
    int per[3];
    double shift[9];
};

// Coordinate c at lattice point q; on periodic axes q may be outside [0,n) and
// each crossed period adds the period shift (periodic extension of the grid).
__device__ double coord_at(const CoordGrid &G, int c, int q0, int q1, int q2)
{
    int q[3] = {q0, q1, q2};
    double off = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (G.per[a]) {
            int w = floordiv_i(q[a], G.n[a]);
            q[a] -= w * G.n[a];
            off += w * G.shift[3 * a + c];
        }
    }
    return G.X[c][((long long)q[2] * G.n[1] + q[1]) * G.n[0] + q[0]] + off;
}

// The metric stencils use explicitly rounded products and sums (no FMA
// contraction): on a Cartesian-product grid the cross terms are then exact
// zeros, as they are mathematically.  The boundary conditions branch on the
// sign of the normal velocity, and an edge point whose interior neighbour
// carries zero normal velocity must not see round-off residue there.

// d x_c / d xi^a at lattice point q.
__device__ double dcoord(const CoordGrid &G, int c, int a, const int q[3])
{
    // one-sided stencils are chosen from the wrapped index on periodic axes
    Stencil s = deriv_stencil(q[a], G.n[a], G.per[a]);
    double acc = 0.0;
    for (int t = 0; t < s.n; ++t) {
        int r[3] = {q[0], q[1], q[2]};
        r[a] += s.off[t];
        acc = __dadd_rn(acc, __dmul_rn(s.wgt[t], coord_at(G, c, r[0], r[1], r[2])));
    }
    return acc;
}

// D_outer [ x_c1 * D_inner x_c2 ] at lattice point q.
__device__ double dprod(const CoordGrid &G, int c1, int c2, int inner, int outer, const int q[3])
{
    Stencil s = deriv_stencil(q[outer], G.n[outer], G.per[outer]);
    double acc = 0.0;
    for (int t = 0; t < s.n; ++t) {
        int r[3] = {q[0], q[1], q[2]};
        r[outer] += s.off[t];
        double prod = __dmul_rn(coord_at(G, c1, r[0], r[1], r[2]), dcoord(G, c2, inner, r));
        acc = __dadd_rn(acc, __dmul_rn(s.wgt[t], prod));
    }
    return acc;
}

__global__ void __launch_bounds__(BLOCK) k_metrics(CoordGrid G, double *met, long long fs,
                                                   int pitch, double Cs)
{
    long long total = (long long)G.n[0] * G.n[1] * G.n[2];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        int q[3];
        q[0] = (int)(p % G.n[0]);
        q[1] = (int)((p / G.n[0]) % G.n[1]);
        q[2] = (int)(p / ((long long)G.n[0] * G.n[1]));
        long long o = ((long long)q[2] * G.n[1] + q[1]) * pitch + q[0];
        // conservative cofactors: J^-1 d xi^a / d x_c =
        //   D_b( x_c1 D_d x_c2 ) - D_d( x_c1 D_b x_c2 ),  (a,b,d), (c,c1,c2) cyclic
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, d = (a + 2) % 3;
            for (int c = 0; c < 3; ++c) {
                int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                met[(3 * a + c) * fs + o] = __dsub_rn(dprod(G, c1, c2, d, b, q), dprod(G, c1, c2, b, d, q));
            }
        }
        double t[3][3];
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) t[c][a] = dcoord(G, c, a, q);
        // determinant of d(x,y,z)/d(xi,eta,zeta), as printed for 1/J
        double m0 = __dsub_rn(__dmul_rn(t[1][1], t[2][2]), __dmul_rn(t[1][2], t[2][1]));
        double m1 = __dsub_rn(__dmul_rn(t[1][0], t[2][2]), __dmul_rn(t[1][2], t[2][0]));
        double m2 = __dsub_rn(__dmul_rn(t[1][0], t[2][1]), __dmul_rn(t[1][1], t[2][0]));
        double jinv = __dadd_rn(__dsub_rn(__dmul_rn(t[0][0], m0), __dmul_rn(t[0][1], m1)),
                                __dmul_rn(t[0][2], m2));
        met[MET_JINV * fs + o] = jinv;
        double delta = cbrt(jinv); // filter width: cube root of the cell volume
        met[MET_CSD2 * fs + o] = (Cs * delta) * (Cs * delta);
    }
}

// General FP32 form: the 15 static fields the fused stage reads per point,
// packed into four consecutive float4 records so that the load phase fetches
// them with four vector loads from one array instead of fifteen.
// Separable form on a Cartesian-product grid: the spacing h_a(q) = d x_a /
// d xi^a along each axis, by the same FP64 stencils as the metrics (on such a
// grid the cofactors are products of these), stored with 1/h_a and h_a^(2/3)
// in FP32 for the fused stage.
__global__ void __launch_bounds__(BLOCK) k_sep_metrics(CoordGrid G, float4 *h1x, float4 *h1y, float4 *h1z)
{
    const int tot = G.n[0] + G.n[1] + G.n[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        const int a = t < G.n[0] ? 0 : (t < G.n[0] + G.n[1] ? 1 : 2);
        const int qa = a == 0 ? t : (a == 1 ? t - G.n[0] : t - G.n[0] - G.n[1]);
        int q[3] = {0, 0, 0};
        q[a] = qa;
        const double h = dcoord(G, a, a, q);
        const double c = cbrt(h);
        float4 *out = a == 0 ? h1x : (a == 1 ? h1y : h1z);
        out[qa] = make_float4((float)h, (float)(1.0 / h), (float)(c * c), 0.0f);
    }
}

void launch_sep_metrics(const double *x, const double *y, const double *z, const int n[3], const int per[3],
                        const double shift[9], float4 *h1x, float4 *h1y, float4 *h1z, cudaStream_t st)
{
    CoordGrid G;
    G.X[0] = x;
    G.X[1] = y;
    G.X[2] = z;
    for (int a = 0; a < 3; ++a) {
        G.n[a] = n[a];
        G.per[a] = per[a];
    }
    for (int t = 0; t < 9; ++t) G.shift[t] = shift[t];
    const int tot = n[0] + n[1] + n[2];
    k_sep_metrics<<<(tot + BLOCK - 1) / BLOCK, BLOCK, 0, st>>>(G, h1x, h1y, h1z);
}

// Static per-point fields derived from the metrics (FP64): J = 1/J^-1; per
// axis a the interface average of J^-1 towards the +a neighbour, its
// reciprocal, and the norm of metric row a.
__global__ void __launch_bounds__(BLOCK) k_static_fields(double *met, long long fs, int pitch, int ni,
                                                         int nj, int nk, int p0, int p1, int p2,
                                                         int iface_tables)
{
    const int n[3] = {ni, nj, nk};
    const int per[3] = {p0, p1, p2};
    const long long total = (long long)ni * nj * nk;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        int q[3];
        q[0] = (int)(p % ni);
        q[1] = (int)((p / ni) % nj);
        q[2] = (int)(p / ((long long)ni * nj));
        const long long o = ((long long)q[2] * nj + q[1]) * pitch + q[0];
        const double jinv = met[MET_JINV * fs + o];
        met[MET_J * fs + o] = 1.0 / state_scale(jinv);
        for (int a = 0; a < 3; ++a) {
            int r[3] = {q[0], q[1], q[2]};
            if (per[a]) r[a] = (q[a] + 1) % n[a];
            else if (q[a] + 1 < n[a]) r[a] = q[a] + 1;
            const long long oR = ((long long)r[2] * nj + r[1]) * pitch + r[0];
            const double jb = 0.5 * (jinv + met[MET_JINV * fs + oR]);
            // stored halved: the interface flux wants 1/2 (sum of the two
            // points' coefficients) times J^-1, so the 1/2 is taken here once
            met[(MET_JB + a) * fs + o] = 0.5 * jb;
            // an interface along the degenerate axis has no volume: zero weights
            met[(MET_RJB + a) * fs + o] = jb > 0.0 ? 1.0 / jb : 0.0;
            const double mx = met[(3 * a) * fs + o], my = met[(3 * a + 1) * fs + o],
                         mz = met[(3 * a + 2) * fs + o];
            met[(MET_NORM + a) * fs + o] = sqrt(mx * mx + my * my + mz * mz);
            if (iface_tables) {
                const double rjb = jb > 0.0 ? 1.0 / jb : 0.0;
                double A[9];
                for (int b = 0; b < 3; ++b)
                    for (int c = 0; c < 3; ++c) {
                        const double mc = 0.5 * (met[(3 * b + c) * fs + o] + met[(3 * b + c) * fs + oR]);
                        A[3 * b + c] = mc * rjb * (b == a ? 1.0 : 0.5);
                        met[(MET_A0 + 9 * a + 3 * b + c) * fs + o] = A[3 * b + c];
                    }
                for (int b = 0; b < 3; ++b)
                    met[(MET_K0 + 3 * a + b) * fs + o] =
                        A[3 * a] * A[3 * b] + A[3 * a + 1] * A[3 * b + 1] + A[3 * a + 2] * A[3 * b + 2];
            }
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_convert_metrics(const double *met64, long long fs64,
                                                           real *met, long long fs, long long npad)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npad;
         p += (long long)gridDim.x * blockDim.x)
        for (int f = 0; f < NMET; ++f) met[f * fs + p] = (real)met64[f * fs64 + p];
}

// ---------------------------------------------------------------------------
// Boundary conditions (FP64 arithmetic on the stored state)
// ---------------------------------------------------------------------------

struct Prim64 {
    double rho, u[3], p;
};

__device__ __forceinline__ void cons_of(const Prim64 &s, double g, double Q[5])
{
    Q[0] = s.rho;
    Q[1] = s.rho * s.u[0];
    Q[2] = s.rho * s.u[1];
    Q[3] = s.rho * s.u[2];
    Q[4] = s.p / (g - 1.0) + 0.5 * s.rho * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]);
}

__device__ __forceinline__ Prim64 prim_of(const double Q[5], double g)
{
    Prim64 s;
    s.rho = Q[0];
    for (int c = 0; c < 3; ++c) s.u[c] = Q[1 + c] / Q[0];
    s.p = (g - 1.0) * (Q[4] - 0.5 * Q[0] * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]));
    return s;
}

// Primitive state in the arithmetic type T of the boundary pass.
template <typename T> struct PrimT {
    T rho, u[3], p;
};

// Per-jet constants of the boundary arithmetic: 1/(gamma-1), 1/gamma and the
// ambient speed of sound; reciprocals replace the divisions of the formulas
// (FP64 division is a long instruction sequence on this GPU).
template <typename T> struct BcK {
    T g, g1, rg, TR, cinf;
};

template <typename T> __device__ __forceinline__ void cons_t(const PrimT<T> &s, const BcK<T> &k, T Q[5])
{
    Q[0] = s.rho;
    Q[1] = s.rho * s.u[0];
    Q[2] = s.rho * s.u[1];
    Q[3] = s.rho * s.u[2];
    Q[4] = s.p * k.g1 + T(0.5) * s.rho * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]);
}

// Primitives of a conserved vector; rr = 1/rho.
template <typename T> __device__ __forceinline__ PrimT<T> prim_t(const T Q[5], T g, T &rr)
{
    PrimT<T> s;
    s.rho = Q[0];
    rr = T(1) / Q[0];
    for (int c = 0; c < 3; ++c) s.u[c] = Q[1 + c] * rr;
    s.p = (g - T(1)) * (Q[4] - T(0.5) * Q[0] * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]));
    return s;
}


// Far field (Sec. "Far Field Boundary"): Riemann invariants along the unit
// outward normal n; R- from the ambient at rest, R+ from the interior point.
template <typename T>
__device__ void bc_farfield(const BcK<T> &k, const T Qe[5], const T n[3], T Qf[5])
{
    const T g = k.g;
    T rr;
    const PrimT<T> e = prim_t(Qe, g, rr);
    const T pinf = k.rg, rinf = k.TR;
    const T ce2 = g * e.p * rr; // c_e^2
    const T rce = rsqrt(ce2), ce = ce2 * rce;
    const T qne = e.u[0] * n[0] + e.u[1] * n[1] + e.u[2] * n[2];
    const T rp = qne + T(2) * ce * k.g1;
    const T rm = T(0) - T(2) * k.cinf * k.g1;
    const T qnf = T(0.5) * (rp + rm);
    const T cf = T(0.25) * (g - T(1)) * (rp - rm);
    const T mn = qne * rce;
    PrimT<T> f;
    if (mn >= T(1)) {
        for (int t = 0; t < 5; ++t) Qf[t] = Qe[t];
        return;
    }
    if (mn <= T(-1)) {
        f.rho = rinf;
        f.u[0] = f.u[1] = f.u[2] = T(0);
        f.p = pinf;
        cons_t(f, k, Qf);
        return;
    }
    // subsonic outflow, and |M_n| <= 1e-8 (q_n = 0 up to the rounding of weak
    // waves, which the paper's ranges leave open): entropy and tangential
    // velocity from inside
    if (mn >= T(-1e-8)) {
        // rho_f = (rho_e^gamma c_f^2 / (gamma p_e))^(1/(gamma-1)), gamma p_e = rho_e c_e^2
        for (int c = 0; c < 3; ++c) f.u[c] = e.u[c] + (qnf - qne) * n[c];
        f.rho = pow(pow(e.rho, g) * cf * cf * (rr * rce * rce), k.g1);
    } else { // subsonic inflow: from the ambient (q_n,inf = 0, gamma p_inf = 1)
        for (int c = 0; c < 3; ++c) f.u[c] = T(0) + (qnf - T(0)) * n[c];
        f.rho = pow(pow(rinf, g) * cf * cf, k.g1);
    }
    f.p = f.rho * cf * cf * k.rg;
    cons_t(f, k, Qf);
}

// Exit (Sec. "Exit Boundary Condition").
template <typename T> __device__ void bc_exit(const BcK<T> &k, const T Qe[5], const T n[3], T Qf[5])
{
    const T g = k.g;
    T rr;
    const PrimT<T> e = prim_t(Qe, g, rr);
    if ((e.u[0] * n[0] + e.u[1] * n[1] + e.u[2] * n[2]) * rsqrt(g * e.p * rr) >= T(1)) {
        for (int t = 0; t < 5; ++t) Qf[t] = Qe[t];
        return;
    }
    // p_f = p_inf = 1/gamma with the interior internal energy e_i = p/((gamma-1) rho)
    const T ei = e.p * k.g1 * rr;
    const T rho = e.rho / (g * e.p);
    Qf[0] = rho;
    Qf[1] = rho * e.u[0];
    Qf[2] = rho * e.u[1];
    Qf[3] = rho * e.u[2];
    Qf[4] = rho * (ei + T(0.5) * (e.u[0] * e.u[0] + e.u[1] * e.u[1] + e.u[2] * e.u[2]));
}

// FP32 storage: the boundary arithmetic runs in FP32 except the interior
// pressure and the temperature difference T_e - T_inf = c_e^2 - c_inf^2,
// which are formed in FP64 from the stored values.  The far-field face state
// differs from the interior (or ambient) one by small amounts: the normal
// velocity by (c_e - c_inf)/(gamma - 1) - q_n,e/2, the density and pressure by
// factors (c_f/c)^m close to 1.  Each of these is computed as a difference
// that is accurate relative to itself (c_e - c_inf from T_e - T_inf; the
// factors as 1 + expm1(m log1p(x)) with x = c_f/c - 1 formed from small
// terms), so that FP32 rounding does not seed pressure or transverse
// momentum noise on the faces.
struct BcF {
    float g, g1, rg, TR, cinf, e2, e2g; // gamma, 1/(gamma-1), 1/gamma, ambient rho and c,
                                        // 2/(gamma-1), 2 gamma/(gamma-1)
    double gd, gm1d, Tinfd;             // gamma, gamma - 1, ambient T = c_inf^2 = 1/TR
};

__device__ __forceinline__ void cons_f(float rho, const float u[3], float p, const BcF &k, float Q[5])
{
    Q[0] = rho;
    Q[1] = rho * u[0];
    Q[2] = rho * u[1];
    Q[3] = rho * u[2];
    Q[4] = p * k.g1 + 0.5f * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// Far field (Sec. "Far Field Boundary") for FP32 storage.  With
// R+- = q_n +- 2c/(gamma-1) (R- of the ambient at rest, R+ of the interior):
// q_n,f = (R+ + R-)/2 = q_n,e/2 + (c_e - c_inf)/(gamma-1) and
// c_f = (gamma-1)(R+ - R-)/4 = (gamma-1) q_n,e/4 + (c_e + c_inf)/2.  The
// isentropic density rho_e^gamma c_f^2 / (gamma p_e), raised to 1/(gamma-1),
// is rho_e (c_f/c_e)^(2/(gamma-1)) since gamma p_e = rho_e c_e^2, and the face
// pressure rho_f c_f^2 / gamma is p_e (c_f/c_e)^(2 gamma/(gamma-1)); on inflow
// the same with the ambient state (rho_inf c_inf^2 = gamma p_inf = 1).
__device__ void bc_farfield_f32(const BcF &k, const float Qe[5], const float n[3], float Qf[5])
{
    const double rho64 = Qe[0];
    const double rr64 = 1.0 / rho64;
    const double ke2 = ((double)Qe[1] * Qe[1] + (double)Qe[2] * Qe[2] + (double)Qe[3] * Qe[3]) * rr64; // rho |u|^2
    const double p64 = k.gm1d * ((double)Qe[4] - 0.5 * ke2);
    const double T64 = k.gd * p64 * rr64;
    const float dT = (float)(T64 - k.Tinfd); // T_e - T_inf
    const float rr = (float)rr64;
    const float u[3] = {Qe[1] * rr, Qe[2] * rr, Qe[3] * rr};
    const float ce = sqrtf((float)T64);
    const float dc = dT / (ce + k.cinf); // c_e - c_inf
    const float qne = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    const float mn = qne / ce;
    if (mn >= 1.0f) { // supersonic outflow: all from inside
        for (int t = 0; t < 5; ++t) Qf[t] = Qe[t];
        return;
    }
    if (mn <= -1.0f) { // supersonic inflow: the ambient at rest
        const float z[3] = {0.0f, 0.0f, 0.0f};
        cons_f(k.TR, z, k.rg, k, Qf);
        return;
    }
    const float qv = 0.25f * (k.g - 1.0f) * qne; // c_f = qv + (c_e + c_inf)/2
    float uf[3], rho, p;
    // subsonic outflow, and |M_n| <= 1e-8 (as in the FP64 form): entropy and
    // tangential velocity from inside
    if (mn >= -1e-8f) {
        const float dq = k.g1 * dc - 0.5f * qne; // q_n,f - q_n,e
        for (int c = 0; c < 3; ++c) uf[c] = u[c] + dq * n[c];
        const float L = log1pf((qv - 0.5f * dc) / ce); // log(c_f/c_e)
        const float rho_e = Qe[0], p_e = (float)p64;
        rho = fmaf(rho_e, expm1f(k.e2 * L), rho_e);
        p = fmaf(p_e, expm1f(k.e2g * L), p_e);
    } else { // subsonic inflow: from the ambient (q_n,inf = 0)
        const float qnf = 0.5f * qne + k.g1 * dc;
        for (int c = 0; c < 3; ++c) uf[c] = qnf * n[c];
        const float L = log1pf((qv + 0.5f * dc) / k.cinf); // log(c_f/c_inf)
        rho = fmaf(k.TR, expm1f(k.e2 * L), k.TR);
        p = fmaf(k.rg, expm1f(k.e2g * L), k.rg);
    }
    cons_f(rho, uf, p, k, Qf);
}

// Exit (Sec. "Exit Boundary Condition") for FP32 storage (the interior
// pressure, e - rho |u|^2 / 2, in FP64).
__device__ void bc_exit_f32(const BcF &k, const float Qe[5], const float n[3], float Qf[5])
{
    const double rr64 = 1.0 / (double)Qe[0];
    const float rr = (float)rr64;
    const float u[3] = {Qe[1] * rr, Qe[2] * rr, Qe[3] * rr};
    const float q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float p = (float)(k.gm1d * ((double)Qe[4] -
                                      0.5 * ((double)Qe[1] * Qe[1] + (double)Qe[2] * Qe[2] + (double)Qe[3] * Qe[3]) * rr64));
    if ((u[0] * n[0] + u[1] * n[1] + u[2] * n[2]) * rsqrtf(k.g * p * rr) >= 1.0f) {
        for (int t = 0; t < 5; ++t) Qf[t] = Qe[t];
        return;
    }
    // p_f = p_inf = 1/gamma with the interior internal energy p/((gamma-1) rho)
    const float ei = p * k.g1 * rr;
    const float rho = Qe[0] / (k.g * p);
    Qf[0] = rho;
    Qf[1] = rho * u[0];
    Qf[2] = rho * u[1];
    Qf[3] = rho * u[2];
    Qf[4] = rho * (ei + 0.5f * q2);
}

// Centerline (Sec. "Centerline Boundary Condition"): one thread per (axial
// station i, conserved variable f) of a jet whose j- face is the axis sums the
// unscaled ring j = 1 over k in index order (deterministic, the same sum for
// every axis point) and writes the mean, unscaled (state scale 1), to all
// azimuthal copies of the axis point (i, 0, k).
template <typename real>
__global__ void __launch_bounds__(BLOCK) k_centerline(const JetDev<real> *__restrict__ jets, int dst)
{
    const JetDev<real> &J = jets[blockIdx.y];
    if (J.bc[2] != LES_BC_CENTERLINE) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 5 * J.n[0]) return;
    const int i = t / 5, f = t % 5;
    const long long fs = J.fs;
    real *Q = J.q[dst] + f * fs;
    double sum = 0.0;
    for (int k = 0; k < J.n[2]; ++k) {
        const long long o = lidx(J, i, 1, k);
        sum += (double)Q[o] / stored_scale<real>(J.jinv64[o]);
    }
    const double avg = sum / (double)J.n[2];
    for (int k = 0; k < J.n[2]; ++k) Q[lidx(J, i, 0, k)] = (real)avg;
}

// SplitMix64: output number n of the generator seeded with `seed`.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long n)
{
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Inflow noise of velocity component c at face point (jj, kk) for the step
// that `level` counts (level > 0): A U_j (2h - 1), h in [0, 1) the top 53 bits
// of SplitMix64 output number ((level - 1) nk + kk) nj + jj) * 3 + c.
template <typename real>
__device__ __forceinline__ double inflow_noise(const JetDev<real> &J, long long level, int kk, int jj, int c)
{
    const unsigned long long ctr =
        ((((unsigned long long)(level - 1) * (unsigned long long)J.n[2] + (unsigned long long)kk) *
              (unsigned long long)J.n[1] +
          (unsigned long long)jj) * 3ull) + (unsigned long long)c;
    const double h = (double)(splitmix64(J.seed, ctr) >> 11) * (1.0 / 9007199254740992.0);
    return J.noise_amp * J.mach * (2.0 * h - 1.0);
}

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_bc(const JetDev<real> *__restrict__ jets, BlockMap bm,
                                              int axis, int dst, const long long *__restrict__ level_p)
{
    const long long level = *level_p;
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        if (J.per[axis]) continue;
        // tangential axes, the lower one fastest across threads (i on the y
        // and z faces, so those passes read and write whole rows)
        const int b = axis == 0 ? 1 : 0, d = axis == 2 ? 1 : 2;
        const long long nface = (long long)J.n[b] * J.n[d];
        long long t = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        if (t >= 2 * nface) continue;
        const int side = (int)(t / nface);
        const long long r = t - side * nface;
        const int ib = (int)(r % J.n[b]), id = (int)(r / J.n[b]);
        const int type = J.bc[2 * axis + side];
        int qf[3], qe[3];
        qf[axis] = side ? J.n[axis] - 1 : 0;
        qe[axis] = side ? J.n[axis] - 2 : 1;
        qf[b] = qe[b] = ib;
        qf[d] = qe[d] = id;
        const long long F = lidx(J, qf[0], qf[1], qf[2]);
        const long long E = lidx(J, qe[0], qe[1], qe[2]);
        const long long fs = J.fs;
        real *Qd = J.q[dst];
        const int jj = qf[1], kk = qf[2];
        if constexpr (sizeof(real) == sizeof(float)) {
            // FP32 storage: FP32 arithmetic (see bc_farfield_f32)
            const BcF k{(float)J.gamma, (float)J.bc_g1, (float)J.bc_rg, (float)J.TR, (float)J.bc_cinf,
                        (float)(2.0 * J.bc_g1), (float)(2.0 * J.gamma * J.bc_g1), J.gamma, J.gamma - 1.0, 1.0 / J.TR};
            float n[3], nn = 0.0f;
            const float sg = side ? 1.0f : -1.0f;
            for (int c = 0; c < 3; ++c) {
                n[c] = sg * (float)J.met[(3 * axis + c) * fs + F];
                nn += n[c] * n[c];
            }
            const float rn = rsqrtf(nn);
            for (int c = 0; c < 3; ++c) n[c] *= rn;
            float Qe[5], Qf[5];
            for (int f = 0; f < 5; ++f) Qe[f] = (float)Qd[f * fs + E];
            if (type == LES_BC_FARFIELD) {
                bc_farfield_f32(k, Qe, n, Qf);
            } else if (type == LES_BC_EXIT) {
                bc_exit_f32(k, Qe, n, Qf);
            } else if (type == LES_BC_INFLOW_JET) {
                const double utd = J.inflow_ut[(long long)kk * J.n[1] + jj];
                if (utd < 0.01) {
                    bc_farfield_f32(k, Qe, n, Qf);
                } else {
                    const float ut = (float)utd, M = (float)J.mach, g = k.g;
                    float uf[3];
                    float p, rho;
                    if (M < 1.0f) {
                        // subsonic entrance (see the FP64 form below)
                        uf[0] = M * ut;
                        if (level > 0) uf[0] += (float)inflow_noise(J, level, kk, jj, 0);
                        const float rre = 1.0f / Qe[0];
                        uf[1] = Qe[2] * rre;
                        uf[2] = Qe[3] * rre;
                        const float Ttot = 1.0f + 0.5f * (g - 1.0f) * M * M;
                        const float Ts = Ttot / (1.0f + 0.5f * (g - 1.0f) * (uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2]));
                        p = powf(Ts, g * k.g1) * k.rg;
                        rho = g * p / Ts;
                    } else {
                        const float Tt = (1.0f / k.TR) * (1.0f - ut) + ut + 0.5f * (g - 1.0f) * M * M * ut * (1.0f - ut);
                        p = k.rg;
                        rho = 1.0f / Tt; // gamma p / T
                        uf[0] = M * ut;
                        uf[1] = uf[2] = 0.0f;
                        if (level > 0)
                            for (int c = 0; c < 3; ++c) uf[c] += (float)inflow_noise(J, level, kk, jj, c);
                    }
                    cons_f(rho, uf, p, k, Qf);
                }
            } else {
                continue;
            }
            for (int f = 0; f < 5; ++f) Qd[f * fs + F] = (real)Qf[f];
        } else {
        using T = double; // FP64 storage: boundary arithmetic in FP64
        const BcK<T> k{(T)J.gamma, (T)J.bc_g1, (T)J.bc_rg, (T)J.TR, (T)J.bc_cinf};
        const T g = k.g;
        // unit outward normal from the face point's metric row
        T n[3], nn = T(0);
        const T sg = side ? T(1) : T(-1);
        for (int c = 0; c < 3; ++c) {
            n[c] = sg * J.met[(3 * axis + c) * fs + F];
            nn += n[c] * n[c];
        }
        const T rn = rsqrt(nn);
        for (int c = 0; c < 3; ++c) n[c] *= rn;
        const T jinvE = (T)stored_scale<real>(J.jinv64[E]), jinvF = (T)stored_scale<real>(J.jinv64[F]);
        const T rjE = T(1) / jinvE;
        T Qe[5], Qf[5];
        for (int f = 0; f < 5; ++f) Qe[f] = Qd[f * fs + E] * rjE;
        if (type == LES_BC_FARFIELD) {
            bc_farfield<T>(k, Qe, n, Qf);
        } else if (type == LES_BC_EXIT) {
            bc_exit<T>(k, Qe, n, Qf);
        } else if (type == LES_BC_INFLOW_JET) {
            const T ut = (T)J.inflow_ut[(long long)kk * J.n[1] + jj];
            const T M = (T)J.mach;
            if (ut < T(0.01)) {
                bc_farfield<T>(k, Qe, n, Qf);
            } else if (M < T(1)) {
                // Sec. "Entrance Boundary", subsonic entrance: u fixed (profile
                // and the u noise of the level), v and w from the interior
                // point, T from the jet's total temperature 1 + (gamma-1) M^2/2
                // with the face velocity in units of a_j, p = T^(gamma/(gamma-1))/gamma
                T u = M * ut;
                if (level > 0) u += (T)inflow_noise(J, level, kk, jj, 0);
                const T rre = T(1) / Qe[0];
                const T v = Qe[2] * rre, w = Qe[3] * rre;
                const T Ttot = T(1) + T(0.5) * (g - T(1)) * M * M;
                const T Ts = Ttot / (T(1) + T(0.5) * (g - T(1)) * (u * u + v * v + w * w));
                PrimT<T> s;
                s.p = pow(Ts, g * k.g1) * k.rg;
                s.rho = g * s.p / Ts;
                s.u[0] = u;
                s.u[1] = v;
                s.u[2] = w;
                cons_t(s, k, Qf);
            } else {
                const T Tt = (T(1) / (T)J.TR) * (T(1) - ut) + ut + T(0.5) * (g - T(1)) * M * M * ut * (T(1) - ut);
                PrimT<T> s;
                s.p = T(1) / g;
                s.rho = g * s.p / Tt;
                s.u[0] = M * ut;
                s.u[1] = s.u[2] = T(0);
                if (level > 0)
                    for (int c = 0; c < 3; ++c) s.u[c] += (T)inflow_noise(J, level, kk, jj, c);
                cons_t(s, k, Qf);
            }
        } else {
            continue;
        }
        for (int f = 0; f < 5; ++f) Qd[f * fs + F] = (real)(jinvF * Qf[f]);
        }
    }
}

// ---------------------------------------------------------------------------
// State conversion (host dense FP64 <-> device padded Qhat)
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_set_state(const JetDev<real> *__restrict__ jets, int jet,
                                                     const double *__restrict__ in, int kind)
{
    const JetDev<real> &J = jets[jet];
    const long long N = (long long)J.n[0] * J.n[1] * J.n[2];
    for (long long lp = blockIdx.x * (long long)blockDim.x + threadIdx.x; lp < J.npts_pad;
         lp += (long long)gridDim.x * blockDim.x) {
        int q[3];
        if (!point_of(J, lp, q)) continue;
        long long dense = ((long long)q[2] * J.n[1] + q[1]) * J.n[0] + q[0];
        double v[5];
        for (int f = 0; f < 5; ++f) v[f] = in[f * N + dense];
        real *Q = J.q[0];
        if (kind == LES_STATE_RAW) {
            for (int f = 0; f < 5; ++f) Q[f * J.fs + lp] = (real)v[f];
            continue;
        }
        double Qc[5];
        if (kind == LES_STATE_PRIMITIVE) {
            Prim64 s;
            s.rho = v[0];
            s.u[0] = v[1];
            s.u[1] = v[2];
            s.u[2] = v[3];
            s.p = v[4];
            cons_of(s, J.gamma, Qc);
        } else {
            for (int f = 0; f < 5; ++f) Qc[f] = v[f];
        }
        const double jinv = stored_scale<real>(J.jinv64[lp]);
        for (int f = 0; f < 5; ++f) Q[f * J.fs + lp] = (real)(jinv * Qc[f]);
    }
}

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_get_state(const JetDev<real> *__restrict__ jets, int jet,
                                                     double *__restrict__ out, int kind)
{
    const JetDev<real> &J = jets[jet];
    const long long N = (long long)J.n[0] * J.n[1] * J.n[2];
    for (long long lp = blockIdx.x * (long long)blockDim.x + threadIdx.x; lp < J.npts_pad;
         lp += (long long)gridDim.x * blockDim.x) {
        int q[3];
        if (!point_of(J, lp, q)) continue;
        long long dense = ((long long)q[2] * J.n[1] + q[1]) * J.n[0] + q[0];
        const real *Q = J.q[0];
        double v[5];
        for (int f = 0; f < 5; ++f) v[f] = (double)Q[f * J.fs + lp];
        if (kind != LES_STATE_RAW) {
            const double jinv = stored_scale<real>(J.jinv64[lp]);
            for (int f = 0; f < 5; ++f) v[f] /= jinv;
            if (kind == LES_STATE_PRIMITIVE) {
                Prim64 s = prim_of(v, J.gamma);
                v[0] = s.rho;
                v[1] = s.u[0];
                v[2] = s.u[1];
                v[3] = s.u[2];
                v[4] = s.p;
            }
        }
        for (int f = 0; f < 5; ++f) out[f * N + dense] = v[f];
    }
}

// ---------------------------------------------------------------------------
// Time step: max over points of lambda_xi + lambda_eta + lambda_zeta
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_dt_max(const JetDev<real> *__restrict__ jets, BlockMap bm,
                                                  unsigned long long *maxbits)
{
    __shared__ double red[BLOCK];
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        long long lp = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        double val = 0.0;
        int q[3];
        if (lp < J.npts_pad && point_of(J, lp, q)) {
            const long long fs = J.fs;
            double rj = 1.0 / state_scale((double)J.met[MET_JINV * fs + lp]);
            double u = J.prim[P_U * fs + lp], v = J.prim[P_V * fs + lp], w = J.prim[P_W * fs + lp];
            double c = sqrt((double)J.prim[P_T * fs + lp]);
            for (int a = 0; a < 3; ++a) {
                double mx = J.met[(3 * a) * fs + lp], my = J.met[(3 * a + 1) * fs + lp],
                       mz = J.met[(3 * a + 2) * fs + lp];
                val += fabs((mx * u + my * v + mz * w) * rj) + c * sqrt(mx * mx + my * my + mz * mz) * rj;
            }
        }
        red[threadIdx.x] = val;
        __syncthreads();
        for (int s = BLOCK / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0)
            atomicMax(maxbits + jet, (unsigned long long)__double_as_longlong(red[0]));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Diagnostics: per-block partials in a fixed order, then one block combines.
// partial layout (NPART = 17 doubles): [0] max|RHS_rho|, [1..5] sum RHS^2,
// [6..10] Neumaier sums of Qhat, [11..15] their compensations, [16] the
// count of non-finite state or residual values (reported as out[11]).
// ---------------------------------------------------------------------------

constexpr int NPART = 17;

__device__ __forceinline__ void neumaier_add(double &s, double &c, double v)
{
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_diag_partials(const JetDev<real> *__restrict__ jets,
                                                         int jet, double *partials)
{
    const JetDev<real> &J = jets[jet];
    __shared__ double sh[NPART][BLOCK];
    double mx = 0.0, l2[5] = {0, 0, 0, 0, 0}, s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
    double bad = 0.0;
    const long long fs = J.fs;
    for (long long lp = blockIdx.x * (long long)blockDim.x + threadIdx.x; lp < J.npts_pad;
         lp += (long long)gridDim.x * blockDim.x) {
        int q[3];
        if (!point_of(J, lp, q)) continue;
        // the Qhat the FP64 store holds (unscaled on a polar axis) from an
        // unscaled FP32 store
        const double qs = sizeof(real) == sizeof(float) ? state_scale(J.jinv64[lp]) : 1.0;
        for (int f = 0; f < 5; ++f) {
            double r = (double)J.rhs[f * fs + lp];
            double v = (double)J.q[0][f * fs + lp] * qs;
            if (!isfinite(r) || !isfinite(v)) bad += 1.0;
            l2[f] += r * r;
            neumaier_add(s[f], c[f], v);
        }
        mx = fmax(mx, fabs((double)J.rhs[lp]));
    }
    sh[0][threadIdx.x] = mx;
    for (int f = 0; f < 5; ++f) {
        sh[1 + f][threadIdx.x] = l2[f];
        sh[6 + f][threadIdx.x] = s[f];
        sh[11 + f][threadIdx.x] = c[f];
    }
    sh[16][threadIdx.x] = bad;
    __syncthreads();
    for (int st = BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            int o = threadIdx.x + st;
            sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][o]);
            for (int f = 0; f < 5; ++f) {
                sh[1 + f][threadIdx.x] += sh[1 + f][o];
                double a = sh[6 + f][threadIdx.x], ca = sh[11 + f][threadIdx.x];
                neumaier_add(a, ca, sh[6 + f][o]);
                sh[6 + f][threadIdx.x] = a;
                sh[11 + f][threadIdx.x] = ca + sh[11 + f][o];
            }
            sh[16][threadIdx.x] += sh[16][o];
        }
        __syncthreads();
    }
    if (threadIdx.x < NPART) partials[blockIdx.x * NPART + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_diag_final(const double *partials, int nblocks, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mx = 0.0, l2[5] = {0, 0, 0, 0, 0}, s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0}, bad = 0;
    for (int b = 0; b < nblocks; ++b) {
        const double *P = partials + b * NPART;
        mx = fmax(mx, P[0]);
        for (int f = 0; f < 5; ++f) {
            l2[f] += P[1 + f];
            neumaier_add(s[f], c[f], P[6 + f]);
            c[f] += P[11 + f];
        }
        bad += P[16];
    }
    out[0] = mx;
    for (int f = 0; f < 5; ++f) {
        out[1 + f] = sqrt(l2[f]);
        out[6 + f] = s[f] + c[f];
    }
    out[11] = bad;
}

// ---------------------------------------------------------------------------
// Debug point fields
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_debug_field(const JetDev<real> *__restrict__ jets, int jet,
                                                       int field, double *out)
{
    const JetDev<real> &J = jets[jet];
    const long long N = (long long)J.n[0] * J.n[1] * J.n[2];
    for (long long lp = blockIdx.x * (long long)blockDim.x + threadIdx.x; lp < J.npts_pad;
         lp += (long long)gridDim.x * blockDim.x) {
        int q[3];
        if (!point_of(J, lp, q)) continue;
        long long dense = ((long long)q[2] * J.n[1] + q[1]) * J.n[0] + q[0];
        const long long fs = J.fs;
        switch (field) {
        case LES_FIELD_MU_SGS: out[dense] = J.grad[G_MUSGS * fs + lp]; break;
        case LES_FIELD_MU: out[dense] = J.prim[P_MU * fs + lp]; break;
        case LES_FIELD_P: out[dense] = J.prim[P_P * fs + lp]; break;
        case LES_FIELD_T: out[dense] = J.prim[P_T * fs + lp]; break;
        case LES_FIELD_LAMBDA_XI: out[dense] = J.prim[P_LXI * fs + lp]; break;
        case LES_FIELD_LAMBDA_ETA: out[dense] = J.prim[P_LETA * fs + lp]; break;
        case LES_FIELD_LAMBDA_ZETA: out[dense] = J.prim[P_LZETA * fs + lp]; break;
        case DBG_RHS:
            for (int f = 0; f < NF; ++f) out[f * N + dense] = J.rhs[f * fs + lp];
            break;
        default:
            if (field >= DBG_MET0 && field < DBG_MET0 + 9) out[dense] = J.met[(field - DBG_MET0) * fs + lp];
            else if (field == DBG_MET0 + 9) out[dense] = J.jinv64[lp];
            break;
        }
    }
}

// ---------------------------------------------------------------------------
// Surface probe: trilinear interpolation of rho, u, v, w, p
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_probe(const JetDev<real> *__restrict__ jets,
                                                 const int *__restrict__ cell,
                                                 const double *__restrict__ wts, int npts, int every,
                                                 const long long *__restrict__ level_p,
                                                 const long long *__restrict__ base_p, real *out,
                                                 int capacity)
{
    const long long level = *level_p;
    if (level % every != 0) return;
    const long long frame = level / every - *base_p - 1;
    if (frame < 0) return;
    const JetDev<real> &J = jets[0];
    const long long fs = J.fs;
    real *o = out + (frame % capacity) * 5LL * npts;
    const double g = J.gamma;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < npts; s += gridDim.x * blockDim.x) {
        int lo[3] = {cell[3 * s], cell[3 * s + 1], cell[3 * s + 2]};
        double t[3] = {wts[3 * s], wts[3 * s + 1], wts[3 * s + 2]};
        double acc[5] = {0, 0, 0, 0, 0};
        for (int c = 0; c < 8; ++c) {
            int r[3];
            double wgt = 1.0;
            for (int a = 0; a < 3; ++a) {
                int up = (c >> a) & 1;
                r[a] = lo[a] + up;
                wgt *= up ? t[a] : 1.0 - t[a];
            }
            long long p = lidx(J, r[0], r[1], r[2]);
            double jinv = stored_scale<real>(J.jinv64[p]);
            double Q[5];
            for (int f = 0; f < 5; ++f) Q[f] = (double)J.q[0][f * fs + p] / jinv;
            Prim64 pr = prim_of(Q, g);
            acc[0] += wgt * pr.rho;
            acc[1] += wgt * pr.u[0];
            acc[2] += wgt * pr.u[1];
            acc[3] += wgt * pr.u[2];
            acc[4] += wgt * pr.p;
        }
        for (int f = 0; f < 5; ++f) o[(long long)f * npts + s] = (real)acc[f];
    }
}

__global__ void k_step_advance(long long *level) { *level += 1; }

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static int grid_for(long long work, int cap = 152 * 16)
{
    long long g = (work + BLOCK - 1) / BLOCK;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename real>
void Launch<real>::metrics(const double *x, const double *y, const double *z, int ni, int nj, int nk,
                           const int per[3], const double shift[9], double *met64, long long fs64,
                           int pitch, double Cs, cudaStream_t st)
{
    CoordGrid G;
    G.X[0] = x;
    G.X[1] = y;
    G.X[2] = z;
    G.n[0] = ni;
    G.n[1] = nj;
    G.n[2] = nk;
    for (int a = 0; a < 3; ++a) G.per[a] = per[a];
    for (int t = 0; t < 9; ++t) G.shift[t] = shift[t];
    k_metrics<<<grid_for((long long)ni * nj * nk), BLOCK, 0, st>>>(G, met64, fs64, pitch, Cs);
}

template <typename real>
void Launch<real>::static_fields(double *met64, long long fs64, int pitch, const int n[3],
                                 const int per[3], int iface_tables, cudaStream_t st)
{
    k_static_fields<<<grid_for((long long)n[0] * n[1] * n[2]), BLOCK, 0, st>>>(
        met64, fs64, pitch, n[0], n[1], n[2], per[0], per[1], per[2], iface_tables);
}

template <typename real>
void Launch<real>::convert_metrics(const double *met64, long long fs64, real *met, long long fs,
                                   long long npad, cudaStream_t st)
{
    k_convert_metrics<real><<<grid_for(npad), BLOCK, 0, st>>>(met64, fs64, met, fs, npad);
}

template <typename real>
void launch_centerline(const JetDev<real> *jets, int njets, int max_ni, int dst, cudaStream_t st)
{
    dim3 grid((5 * max_ni + BLOCK - 1) / BLOCK, njets);
    k_centerline<real><<<grid, BLOCK, 0, st>>>(jets, dst);
}
template void launch_centerline<float>(const JetDev<float> *, int, int, int, cudaStream_t);
template void launch_centerline<double>(const JetDev<double> *, int, int, int, cudaStream_t);

template <typename real>
void Launch<real>::bc(const JetDev<real> *jets, BlockMap bm, int axis, int dst,
                      const long long *level, int grid, cudaStream_t st)
{
    k_bc<real><<<grid, BLOCK, 0, st>>>(jets, bm, axis, dst, level);
}

template <typename real>
void Launch<real>::set_state(const JetDev<real> *jets, int jet, const double *in, int kind,
                             long long npad, cudaStream_t st)
{
    k_set_state<real><<<grid_for(npad), BLOCK, 0, st>>>(jets, jet, in, kind);
}

template <typename real>
void Launch<real>::get_state(const JetDev<real> *jets, int jet, double *out, int kind,
                             long long npad, cudaStream_t st)
{
    k_get_state<real><<<grid_for(npad), BLOCK, 0, st>>>(jets, jet, out, kind);
}

template <typename real>
void Launch<real>::dt_max(const JetDev<real> *jets, BlockMap bm, unsigned long long *maxbits,
                          int grid, cudaStream_t st)
{
    k_dt_max<real><<<grid, BLOCK, 0, st>>>(jets, bm, maxbits);
}

template <typename real>
void Launch<real>::diag_partials(const JetDev<real> *jets, int jet, double *partials, int nblocks,
                                 cudaStream_t st)
{
    k_diag_partials<real><<<nblocks, BLOCK, 0, st>>>(jets, jet, partials);
}

template <typename real>
void Launch<real>::debug_field(const JetDev<real> *jets, int jet, int field, double *out,
                               long long npad, cudaStream_t st)
{
    k_debug_field<real><<<grid_for(npad), BLOCK, 0, st>>>(jets, jet, field, out);
}

template <typename real>
void Launch<real>::probe(const JetDev<real> *jets, const int *cell, const double *wts, int npts,
                         int every, const long long *level, const long long *base, real *out,
                         int capacity, cudaStream_t st)
{
    k_probe<real><<<grid_for(npts, 1024), BLOCK, 0, st>>>(jets, cell, wts, npts, every, level, base,
                                                          out, capacity);
}

void launch_diag_final(const double *partials, int nblocks, double *out, cudaStream_t st)
{
    k_diag_final<<<1, 32, 0, st>>>(partials, nblocks, out);
}

void launch_step_advance(long long *level, cudaStream_t st) { k_step_advance<<<1, 1, 0, st>>>(level); }

template struct Launch<float>;
template struct Launch<double>;

} // namespace les
