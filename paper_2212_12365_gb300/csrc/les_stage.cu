// Runge-Kutta stage kernels (Sec. "Time Marching Method", Eq. localdt) of
// libles.so.  One stage runs as four persistent grid-stride kernels:
//   k_point  : per point — primitives from Qhat (EOS, Sec. "Large Eddy
//              Simulation Formulation"), Sutherland mu(T), spectral radii and
//              the anisotropic scaling lambda-bar (Sec. "Numerical
//              Formulation"), the dissipation vector W = Q + [0,0,0,0,p] and
//              the inviscid point fluxes E_e, F_e, G_e (Eq. hat-flux-G)
//   k_grads  : per point — second-order derivatives of u, v, w, T along the
//              three grid axes, the Smagorinsky eddy viscosity and Eidson
//              conductivity (Sec. "Subgrid Scale Modeling"), the pressure
//              sensor per axis (Eq. p_grad_sensor)
//   k_iface  : per interface (one thread owns the +1/2 interfaces of its
//              point along the three axes) — centred inviscid flux minus the
//              Turkel-Vatsa dissipation J^-1 d (Eqs. inv_flux_vec,
//              dissip_term, eps_2/4_dissip) minus the compact viscous + SGS
//              flux (Eqs. hat-flux-Ev/Fv/Gv)
//   k_update : per interior point — the flux differences (Eq. for RHS with
//              Delta xi = 1) and Q(l) = Q(0) - alpha_l dt RHS
// Each interface flux is evaluated once, so the residual of a periodic
// direction telescopes exactly.  On GB300 the FP64 form is bound by the FP64
// pipe, not by HBM: the intermediate fields cost bandwidth that is otherwise
// idle and remove recomputation (divisions, square roots) from the hot loop.
#include <cmath>

#include "les_internal.cuh"

namespace les {

__constant__ double c_alpha[5] = {0.25, 1.0 / 6.0, 0.375, 0.5, 1.0};

// Reciprocal.  FP32 uses the hardware division.  In FP64, whose pipe is the
// bottleneck on this GPU, the reciprocal is a Newton-Raphson iteration
// r <- r (2 - b r) from the hardware's approximate FP64 reciprocal (a seed of
// about single precision, taken without converting through FP32): each step
// squares the relative error, so two steps reach double rounding (a unit in
// the last place) at fewer FP64 operations than an IEEE division, and one
// step leaves a relative error near 1e-14, which is all a factor needs whose
// own error enters the residual damped by its small weight (pressure sensor,
// Sutherland law).  Arguments are positive normal numbers (densities,
// temperatures, sensor denominators).  Square roots stay the native ones (an
// iteration from a single-precision seed measured slower, and must
// special-case zero strain).
__device__ __forceinline__ double rcp_seed(double b)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
    return r;
}
template <typename real> __device__ __forceinline__ real rcp_(real b) { return real(1) / b; }
template <> __device__ __forceinline__ double rcp_<double>(double b)
{
    double r = rcp_seed(b);
    double e = fma(-b, r, 1.0);
    r = fma(r, e, r);
    e = fma(-b, r, 1.0);
    return fma(r, e, r);
}
template <typename real> __device__ __forceinline__ real rcp1_(real b) { return real(1) / b; }
template <> __device__ __forceinline__ double rcp1_<double>(double b)
{
    const double r = rcp_seed(b);
    return fma(r, fma(-b, r, 1.0), r);
}

// ---------------------------------------------------------------------------
// k_point
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_point(const JetDev<real> *__restrict__ jets, BlockMap bm,
                                                 int src)
{
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        const int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        const long long lp = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        int q[3];
        if (lp >= J.npts_pad || !point_of(J, lp, q)) continue;
        const long long fs = J.fs;
        const real *__restrict__ Q = J.q[src];
        const real *__restrict__ M = J.met;
        real *__restrict__ P = J.prim;
        const real gam = (real)J.gamma;
        const real rj = M[MET_J * fs + lp];
        // the stored state times rq is Q: J for a Qhat store, 1 for an
        // unscaled FP32 store
        const real rq = sizeof(real) == sizeof(float) ? real(1) : rj;
        const real rho = Q[lp] * rq;
        const real ru = Q[fs + lp] * rq, rv = Q[2 * fs + lp] * rq, rw = Q[3 * fs + lp] * rq;
        const real e = Q[4 * fs + lp] * rq;
        const real rrho = rcp_<real>(rho);
        const real u = ru * rrho, v = rv * rrho, w = rw * rrho;
        // gamma - 1 and 1 + S from the stored FP64 constants (the values this
        // pass would form; the FP32 instantiation keeps its own rounding)
        const bool f64 = sizeof(real) == sizeof(double);
        const real gm1 = f64 ? (real)J.gm1 : gam - real(1);
        const real p = gm1 * (e - real(0.5) * (ru * u + rv * v + rw * w));
        const real T = gam * p * rrho;
        const real sT = sqrt(T); // speed of sound: c^2 = gamma p / rho = T in jet units
        const real S = (real)J.suth_S;
        const real mu = T * sT * (f64 ? (real)J.suth1 : real(1) + S) * rcp1_<real>(T + S);
        const real rH = e + p;
        real lam[3];
        const real hp = real(0.5) * p;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const real mx = M[(3 * a) * fs + lp], my = M[(3 * a + 1) * fs + lp],
                       mz = M[(3 * a + 2) * fs + lp];
            const real JU = mx * u + my * v + mz * w; // J^-1 times the contravariant velocity
            lam[a] = (fabs(JU) + sT * M[(MET_NORM + a) * fs + lp]) * rj;
            // half the inviscid point flux: the interface average is the sum
            // of the two points' halves
            const real hJU = real(0.5) * JU;
            real *F = P + (P_F0 + 5 * a) * fs + lp;
            F[0] = rho * hJU;
            F[fs] = ru * hJU + hp * mx;
            F[2 * fs] = rv * hJU + hp * my;
            F[3 * fs] = rw * hJU + hp * mz;
            F[4 * fs] = rH * hJU;
        }
        // lambda_a + (lambda_a lambda_b)^1/2 + (lambda_a lambda_d)^1/2 = s_a (s_a + s_b + s_d)
        const real sq0 = sqrt(lam[0]), sq1 = sqrt(lam[1]), sq2 = sqrt(lam[2]);
        const real ssum = sq0 + sq1 + sq2;
        P[P_RHO * fs + lp] = rho;
        P[P_U * fs + lp] = u;
        P[P_V * fs + lp] = v;
        P[P_W * fs + lp] = w;
        P[P_P * fs + lp] = p;
        P[P_T * fs + lp] = T;
        P[P_MU * fs + lp] = mu;
        // lambda-bar_a = lambda_a [1 + (lambda_b/lambda_a)^1/2 + (lambda_d/lambda_a)^1/2]
        P[P_LXI * fs + lp] = sq0 * ssum;
        P[P_LETA * fs + lp] = sq1 * ssum;
        P[P_LZETA * fs + lp] = sq2 * ssum;
        P[P_RU * fs + lp] = ru;
        P[P_RV * fs + lp] = rv;
        P[P_RW * fs + lp] = rw;
        P[P_RH * fs + lp] = rH;
    }
}

// ---------------------------------------------------------------------------
// k_grads
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_grads(const JetDev<real> *__restrict__ jets, BlockMap bm)
{
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        const int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        const long long lp = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        int q[3];
        if (lp >= J.npts_pad || !point_of(J, lp, q)) continue;
        const long long fs = J.fs;
        const real *__restrict__ P = J.prim;
        const real *__restrict__ M = J.met;
        real *__restrict__ G = J.grad;
        real d[4][3]; // d phi / d xi^a, phi = u, v, w, T
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Stencil s = deriv_stencil(q[a], J.n[a], J.per[a]);
            long long o[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                int r[3] = {q[0], q[1], q[2]};
                r[a] = J.per[a] ? wrapi(r[a] + s.off[t], J.n[a]) : r[a] + s.off[t];
                o[t] = lidx(J, r[0], r[1], r[2]);
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const real *F = P + (f < 3 ? P_U + f : P_T) * fs;
                real acc = (real)s.wgt[0] * F[o[0]] + (real)s.wgt[1] * F[o[1]];
                if (s.n == 3) acc += (real)s.wgt[2] * F[o[2]];
                d[f][a] = acc;
            }
            // pressure sensor along a; an end point of a non-periodic axis
            // takes the sensor of its interior neighbour
            int c = q[a];
            if (!J.per[a]) c = c < 1 ? 1 : (c > J.n[a] - 2 ? J.n[a] - 2 : c);
            int rm[3] = {q[0], q[1], q[2]}, r0[3] = {q[0], q[1], q[2]}, rp[3] = {q[0], q[1], q[2]};
            r0[a] = c;
            rm[a] = J.per[a] ? wrapi(c - 1, J.n[a]) : c - 1;
            rp[a] = J.per[a] ? wrapi(c + 1, J.n[a]) : c + 1;
            const real pm = P[P_P * fs + lidx(J, rm[0], rm[1], rm[2])];
            const real p0 = P[P_P * fs + lidx(J, r0[0], r0[1], r0[2])];
            const real pp = P[P_P * fs + lidx(J, rp[0], rp[1], rp[2])];
            const real ps = pp + pm;
            G[(G_NU + a) * fs + lp] = fabs(fma(real(-2), p0, ps)) * rcp1_<real>(fma(real(2), p0, ps));
        }
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int a = 0; a < 3; ++a) G[(3 * f + a) * fs + lp] = d[f][a];
        real m[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) m[t] = M[t * fs + lp];
        const real rj = M[MET_J * fs + lp];
        // d u_i / d x_c = J g_ic with g_ic = sum_b m_bc d u_i / d xi^b (chain
        // rule through the metric cofactors); 2 S_ij S_ij = J^2 (2 sum_i g_ii^2
        // + sum_{i<c} (g_ic + g_ci)^2)
        real g[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) g[i][c] = m[c] * d[i][0] + m[3 + c] * d[i][1] + m[6 + c] * d[i][2];
        real sd = real(0), so = real(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            sd += g[i][i] * g[i][i];
#pragma unroll
            for (int c = i + 1; c < 3; ++c) {
                const real t = g[i][c] + g[c][i];
                so += t * t;
            }
        }
        // Smagorinsky: mu_sgs = rho (Cs Delta)^2 (2 S_ij S_ij)^1/2
        const real mus = P[P_RHO * fs + lp] * M[MET_CSD2 * fs + lp] * rj * sqrt(real(2) * sd + so);
        const real mu = P[P_MU * fs + lp];
        G[G_MUSGS * fs + lp] = mus;
        G[G_MUEFF * fs + lp] = mu * (real)J.inv_Re + mus;
        // Eidson: k_sgs = mu_sgs Cp / Pr_sgs; molecular k = mu Cp / (Re Pr), Cp = 1/(gamma-1)
        G[G_KAP * fs + lp] = mu * (real)J.kap_mol + mus * (real)J.kap_sgs;
    }
}

// ---------------------------------------------------------------------------
// k_iface: flux through the interface between L and R = L + e_a
// ---------------------------------------------------------------------------

// The axis is a template parameter so that every metric/derivative index is a
// compile-time constant (no local-memory arrays).
template <typename real, int a>
__device__ __forceinline__ void iface_flux(const JetDev<real> &J, const int qL[3], long long L,
                                           real *__restrict__ H)
{
    const long long fs = J.fs;
    const real *__restrict__ P = J.prim;
    const real *__restrict__ G = J.grad;
    const real *__restrict__ M = J.met;
    int qR[3] = {qL[0], qL[1], qL[2]};
    qR[a] = J.per[a] ? wrapi(qL[a] + 1, J.n[a]) : qL[a] + 1;
    const long long R = lidx(J, qR[0], qR[1], qR[2]);
    const bool lo_end = !J.per[a] && qL[a] == 0;
    const bool hi_end = !J.per[a] && qR[a] == J.n[a] - 1;
    long long Lm = L, Rp = R;
    if (!lo_end) {
        int r[3] = {qL[0], qL[1], qL[2]};
        r[a] = J.per[a] ? wrapi(qL[a] - 1, J.n[a]) : qL[a] - 1;
        Lm = lidx(J, r[0], r[1], r[2]);
    }
    if (!hi_end) {
        int r[3] = {qR[0], qR[1], qR[2]};
        r[a] = J.per[a] ? wrapi(qR[a] + 1, J.n[a]) : qR[a] + 1;
        Rp = lidx(J, r[0], r[1], r[2]);
    }
    // Turkel-Vatsa: eps2 = k2 max(nu_L, nu_R), eps4 = max(0, k4 - eps2),
    // scaled by the interface lambda-bar and J^-1
    const real eps2 = (real)J.k2 * fmax(G[(G_NU + a) * fs + L], G[(G_NU + a) * fs + R]);
    const real eps4 = fmax(real(0), (real)J.k4 - eps2);
    const real jbh = M[(MET_JB + a) * fs + L]; // half the interface J^-1
    const real sc = jbh * (P[(P_LXI + a) * fs + L] + P[(P_LXI + a) * fs + R]);
    const real se4 = sc * eps4;
    // se2 dW - se4 (dW(+3/2) - 2 dW(+1/2) + dW(-1/2)) with the third
    // difference written as W(R+1) - W(L-1) - 3 dW(+1/2): the flux gains
    // se4 (W(R+1) - W(L-1)) + (se2 + 3 se4) (W(L) - W(R))
    const real c2 = fma(real(3), se4, sc * eps2);
    const int wf[5] = {P_RHO, P_RU, P_RV, P_RW, P_RH};
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        const real *W = P + wf[f] * fs;
        const real wL = W[L], wR = W[R];
        // the mirrored difference at a non-periodic end, dW(outside) = -dW(+1/2),
        // is the missing point W(R+1) = W(L) (resp. W(L-1) = W(R))
        const real wRp = hi_end ? wL : W[Rp];
        const real wLm = lo_end ? wR : W[Lm];
        const real *F = P + (P_F0 + 5 * a + f) * fs;
        // centred flux: the sum of the two points' stored half fluxes
        H[f] = fma(c2, wL - wR, fma(se4, wRp - wLm, F[L] + F[R]));
    }
    // compact viscous + SGS flux: normal derivative from the two points,
    // tangential derivatives averaged, coefficients/metrics/velocity averaged.
    // A = interface tables (cofactor average / interface J^-1, 1/2 folded into
    // the tangential rows), so grad phi = sum_b A_b D_b with D_a = phi_R - phi_L
    // and D_b = the sum of the two points' central differences (b != a); the
    // averaged cofactor row a is A_a times the interface J^-1, folded into the
    // transport coefficients.
    const real *__restrict__ A = M + (MET_A0 + 9 * a) * fs + L;
    real D[4][3];
    const int pf[4] = {P_U, P_V, P_W, P_T};
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            D[f][b] = (b == a) ? P[pf[f] * fs + R] - P[pf[f] * fs + L]
                               : G[(3 * f + b) * fs + L] + G[(3 * f + b) * fs + R];
    real Ab[9], K[3];
#pragma unroll
    for (int t = 0; t < 9; ++t) Ab[t] = A[t * fs];
#pragma unroll
    for (int t = 0; t < 3; ++t) K[t] = M[(MET_K0 + 3 * a + t) * fs + L];
    const real *mr = Ab + 3 * a; // averaged cofactor row a / interface J^-1
    // The flux needs only the row-a contraction of the stress tensor,
    //   s_i = sum_c mr_c tau_ci = ch (X_i + Y_i - 2/3 mr_i tr), ch = mu_eff J^-1,
    // with X_i = sum_c mr_c du_i/dx_c = sum_b K_b D_ib,
    //      Y_i = sum_c mr_c du_c/dx_i = sum_b Ab_bi (sum_c mr_c D_cb),
    //      tr  = div u = sum_i sum_b Ab_bi D_ib,
    // and the energy flux sum_c mr_c (tau_cj u_j + kappa dT/dx_c) =
    // s . u_interface + kappa X_T; tau itself is never formed.
    real X[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) X[f] = K[0] * D[f][0] + K[1] * D[f][1] + K[2] * D[f][2];
    real w[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) w[b] = mr[0] * D[0][b] + mr[1] * D[1][b] + mr[2] * D[2][b];
    // one multiply-add chain over the nine products (no zero start)
    real tr = Ab[0] * D[0][0];
#pragma unroll
    for (int t = 1; t < 9; ++t) tr = fma(Ab[3 * (t % 3) + t / 3], D[t / 3][t % 3], tr);
    // interface averages of mu_eff and kappa times J^-1: the sums times jbh
    const real ch = (G[G_MUEFF * fs + L] + G[G_MUEFF * fs + R]) * jbh;
    const real kap = (G[G_KAP * fs + L] + G[G_KAP * fs + R]) * jbh;
    const real ct = ch * tr * real(2.0 / 3.0);
    real sv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const real Y = Ab[i] * w[0] + Ab[3 + i] * w[1] + Ab[6 + i] * w[2];
        sv[i] = ch * (X[i] + Y) - ct * mr[i];
        H[1 + i] -= sv[i];
    }
    // beta = tau u - q, q = -kappa grad T; interface velocity = average:
    // H4 -= 1/2 sum_i (u_i,L + u_i,R) s_i + kappa X_T, as two multiply-adds
    const real su = (P[P_U * fs + L] + P[P_U * fs + R]) * sv[0] + (P[P_V * fs + L] + P[P_V * fs + R]) * sv[1] +
                    (P[P_W * fs + L] + P[P_W * fs + R]) * sv[2];
    H[4] = fma(-kap, X[3], fma(real(-0.5), su, H[4]));
}

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_iface(const JetDev<real> *__restrict__ jets, BlockMap bm)
{
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        const int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        const long long lp = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        int q[3];
        if (lp >= J.npts_pad || !point_of(J, lp, q)) continue;
        const long long fs = J.fs;
        real H[5];
        // no interface beyond the last point of a non-periodic axis
        if (J.per[0] || q[0] < J.n[0] - 1) {
            iface_flux<real, 0>(J, q, lp, H);
#pragma unroll
            for (int f = 0; f < 5; ++f) J.hflux[f * fs + lp] = H[f];
        }
        if (J.per[1] || q[1] < J.n[1] - 1) {
            iface_flux<real, 1>(J, q, lp, H);
#pragma unroll
            for (int f = 0; f < 5; ++f) J.hflux[(5 + f) * fs + lp] = H[f];
        }
        if (J.per[2] || q[2] < J.n[2] - 1) {
            iface_flux<real, 2>(J, q, lp, H);
#pragma unroll
            for (int f = 0; f < 5; ++f) J.hflux[(10 + f) * fs + lp] = H[f];
        }
    }
}

// ---------------------------------------------------------------------------
// k_update: RHS = sum_a H_a(P) - H_a(P - e_a); Q(dst) = Q(0) - alpha dt RHS
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(BLOCK) k_update(const JetDev<real> *__restrict__ jets, BlockMap bm,
                                                  int dst, int stage, const double *__restrict__ dt,
                                                  int rhs_only)
{
    for (int vb = blockIdx.x; vb < bm.total; vb += gridDim.x) {
        const int jet = find_jet(bm, vb);
        const JetDev<real> &J = jets[jet];
        const long long lp = (long long)(vb - bm.start[jet]) * BLOCK + threadIdx.x;
        int q[3];
        if (lp >= J.npts_pad || !point_of(J, lp, q)) continue;
        const long long fs = J.fs;
        if (!interior(J, q)) {
            if (rhs_only)
                for (int f = 0; f < NF; ++f) J.rhs[f * fs + lp] = real(0);
            continue;
        }
        long long back[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int r[3] = {q[0], q[1], q[2]};
            r[a] = J.per[a] ? wrapi(q[a] - 1, J.n[a]) : q[a] - 1;
            back[a] = lidx(J, r[0], r[1], r[2]);
        }
        const real *__restrict__ Hf = J.hflux;
        real R[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            real acc = Hf[f * fs + lp] - Hf[f * fs + back[0]];
#pragma unroll
            for (int a = 1; a < 3; ++a) acc += Hf[(5 * a + f) * fs + lp] - Hf[(5 * a + f) * fs + back[a]];
            R[f] = acc;
        }
        if (rhs_only) {
#pragma unroll
            for (int f = 0; f < NF; ++f) J.rhs[f * fs + lp] = R[f];
        } else {
            const real adt = (real)(c_alpha[stage] * dt[jet]);
            const real *Q0 = J.q[0];
            real *Qd = J.q[dst];
#pragma unroll
            for (int f = 0; f < NF; ++f) Qd[f * fs + lp] = Q0[f * fs + lp] - adt * R[f];
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <typename real>
void Launch<real>::point(const JetDev<real> *jets, BlockMap bm, int src, int grid, cudaStream_t st)
{
    k_point<real><<<grid, BLOCK, 0, st>>>(jets, bm, src);
}

template <typename real>
void Launch<real>::grads(const JetDev<real> *jets, BlockMap bm, int grid, cudaStream_t st)
{
    k_grads<real><<<grid, BLOCK, 0, st>>>(jets, bm);
}

template <typename real>
void Launch<real>::iface(const JetDev<real> *jets, BlockMap bm, int grid, cudaStream_t st)
{
    k_iface<real><<<grid, BLOCK, 0, st>>>(jets, bm);
}

template <typename real>
void Launch<real>::update(const JetDev<real> *jets, BlockMap bm, int dst, int stage, const double *dt,
                          int rhs_only, int grid, cudaStream_t st)
{
    k_update<real><<<grid, BLOCK, 0, st>>>(jets, bm, dst, stage, dt, rhs_only);
}

template void Launch<float>::point(const JetDev<float> *, BlockMap, int, int, cudaStream_t);
template void Launch<double>::point(const JetDev<double> *, BlockMap, int, int, cudaStream_t);
template void Launch<float>::grads(const JetDev<float> *, BlockMap, int, cudaStream_t);
template void Launch<double>::grads(const JetDev<double> *, BlockMap, int, cudaStream_t);
template void Launch<float>::iface(const JetDev<float> *, BlockMap, int, cudaStream_t);
template void Launch<double>::iface(const JetDev<double> *, BlockMap, int, cudaStream_t);
template void Launch<float>::update(const JetDev<float> *, BlockMap, int, int, const double *, int, int,
                                    cudaStream_t);
template void Launch<double>::update(const JetDev<double> *, BlockMap, int, int, const double *, int, int,
                                     cudaStream_t);

} // namespace les
