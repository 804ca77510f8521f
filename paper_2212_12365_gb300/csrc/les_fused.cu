// Fused single-pass Runge-Kutta stage for FP32 storage and arithmetic.
//
// One kernel does what k_point, k_grads, k_iface and k_update do for the FP64
// path (Secs. "Numerical Formulation", "Time Marching Method"), but the
// intermediate per-point and per-interface quantities live in shared memory
// and registers instead of HBM: per stage a point's state, Q(0) and static
// metrics are read and its new state written once.
//
// Tiling.  A CTA of 32 x TY threads owns the grid columns (ib + tx, jb + ty)
// (region R1, one column per thread) and updates the 30 x (TY-2) inner ones
// (1 <= tx <= 30, 1 <= ty <= TY-2).  Every thread evaluates the xi-interface
// to its +i neighbour (the -i one comes from the lane below by a warp
// shuffle), the eta-interface to its +j neighbour (the -j one from shared
// memory) and the zeta-interface to its +k neighbour (the -k one is carried
// in registers while marching along k).  Point data live in a ring of 5
// planes over R2 = R1 plus one column/row on each side, so that derivatives
// — one-sided at a non-periodic end included — of plane k are formed when
// plane k+2 arrives; derivatives, transport coefficients, sensors and
// lambda-bar of R1 are kept for two planes.  The 32 x 8 variant fits two CTAs
// per SM, so the load phase of one overlaps the arithmetic of the other.
// Per loaded plane kL:  load+primitives(kL) | gradients(kL-2) |
// interfaces+update(kL-3).
//
// Work list.  Items (jet, tile x, tile y, k-chunk) are walked by a persistent
// grid in a fixed order; results do not depend on the item order, the chunk
// length or the grid size.
#include <cmath>

#include "les_internal.cuh"

namespace les {

namespace {

constexpr int FX = 32;  // threads along i (one warp per row)
constexpr int NPF = 6;  // point fields in the ring: rho u v w p T
constexpr int NGF = 20; // R1 fields: 12 derivatives, mu_eff, kappa, nu x3, lambda-bar x3
enum { GF_MUEFF = 12, GF_KAP = 13, GF_NU = 14, GF_LAM = 17 };
constexpr int NMF = 10; // R1 metric fields: 9 cofactors, J^-1

__constant__ float c_alpha_f[5] = {0.25f, 1.0f / 6.0f, 0.375f, 0.5f, 1.0f};

template <int TY> struct Geo {
    static constexpr int NT = FX * TY;
    static constexpr int C2X = FX + 2, C2Y = TY + 2, NC2 = C2X * C2Y; // R2: cells [-1, FX] x [-1, TY]
    static constexpr int NC1 = FX * TY;                                // R1: the thread grid
    static constexpr int OFF_PRIM = 0;                          // [5][NPF][NC2]
    static constexpr int OFF_GRAD = OFF_PRIM + 5 * NPF * NC2;   // [2][NGF][NC1]
    static constexpr int OFF_MET = OFF_GRAD + 2 * NGF * NC1;    // [2][NMF][NC1]
    static constexpr int OFF_HY = OFF_MET + 2 * NMF * NC1;      // [5][TY][FX]
    static constexpr int FLOATS = OFF_HY + 5 * TY * FX;
    static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

__device__ __forceinline__ int ring5(int k) { return ((k % 5) + 5) % 5; }
__device__ __forceinline__ int ring2(int k) { return k & 1; } // two's complement: -1 -> 1

// Wrap a global index on a periodic axis; -1 for outside a non-periodic axis.
__device__ __forceinline__ int gidx(int g, int n, int per)
{
    if (per) return wrapi(g, n);
    return (g >= 0 && g < n) ? g : -1;
}

// Flux through the interface between L and R along axis A.  Smem index
// arguments: p* index the point ring (cell + slot offset), g* the R1 tables.
template <int A, int TY>
__device__ __forceinline__ void fused_iface(const float *__restrict__ S, const FusedParams &FP,
                                            int pLm, int pL, int pR, int pRp, int gL, int gR, int mLi,
                                            int mRi, bool lo_end, bool hi_end, float H[5])
{
    using G_ = Geo<TY>;
    const float *SP = S + G_::OFF_PRIM;
    const float *SG = S + G_::OFF_GRAD;
    const float *SM = S + G_::OFF_MET;
    constexpr int N2 = G_::NC2, N1 = G_::NC1;
    const float hg = FP.hgam;
    // dissipation vector W = [rho, rho u, rho v, rho w, e + p] at the four points
    float W[4][5];
    const int pts[4] = {lo_end ? pL : pLm, pL, pR, hi_end ? pR : pRp};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int o = pts[t];
        const float r = SP[o], u = SP[N2 + o], v = SP[2 * N2 + o], w = SP[3 * N2 + o], p = SP[4 * N2 + o];
        W[t][0] = r;
        W[t][1] = r * u;
        W[t][2] = r * v;
        W[t][3] = r * w;
        W[t][4] = hg * p + 0.5f * r * (u * u + v * v + w * w);
    }
    const float pLv = SP[4 * N2 + pL], pRv = SP[4 * N2 + pR];
    // metric rows at L and R
    float mL[9], mR[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        mL[t] = SM[t * N1 + mLi];
        mR[t] = SM[t * N1 + mRi];
    }
    const float jL = SM[9 * N1 + mLi], jR = SM[9 * N1 + mRi];
    const float jb = 0.5f * (jL + jR);
    const float rjb = 1.0f / jb;
    // centred inviscid flux 0.5 (F_L + F_R), J^-1 U = m_A . u
    {
        const float JUL = mL[3 * A] * SP[N2 + pL] + mL[3 * A + 1] * SP[2 * N2 + pL] + mL[3 * A + 2] * SP[3 * N2 + pL];
        const float JUR = mR[3 * A] * SP[N2 + pR] + mR[3 * A + 1] * SP[2 * N2 + pR] + mR[3 * A + 2] * SP[3 * N2 + pR];
        H[0] = 0.5f * (W[1][0] * JUL + W[2][0] * JUR);
        H[1] = 0.5f * (W[1][1] * JUL + pLv * mL[3 * A] + W[2][1] * JUR + pRv * mR[3 * A]);
        H[2] = 0.5f * (W[1][2] * JUL + pLv * mL[3 * A + 1] + W[2][2] * JUR + pRv * mR[3 * A + 1]);
        H[3] = 0.5f * (W[1][3] * JUL + pLv * mL[3 * A + 2] + W[2][3] * JUR + pRv * mR[3 * A + 2]);
        H[4] = 0.5f * (W[1][4] * JUL + W[2][4] * JUR);
    }
    // Turkel-Vatsa dissipation
    {
        const float eps2 = FP.k2 * fmaxf(SG[(GF_NU + A) * N1 + gL], SG[(GF_NU + A) * N1 + gR]);
        const float eps4 = fmaxf(0.0f, FP.k4 - eps2);
        const float sc = jb * 0.5f * (SG[(GF_LAM + A) * N1 + gL] + SG[(GF_LAM + A) * N1 + gR]);
        const float se2 = sc * eps2, se4 = sc * eps4;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            const float dW0 = W[2][f] - W[1][f];
            const float dWp = hi_end ? -dW0 : W[3][f] - W[2][f];
            const float dWm = lo_end ? -dW0 : W[1][f] - W[0][f];
            const float d3 = dWp - 2.0f * dW0 + dWm;
            H[f] -= se2 * dW0 - se4 * d3;
        }
    }
    // compact viscous + SGS flux
    {
        const int pf[4] = {1, 2, 3, 5}; // u v w T in the point ring
        float dphi[4][3];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                dphi[f][b] = (b == A) ? SP[pf[f] * N2 + pR] - SP[pf[f] * N2 + pL]
                                      : 0.5f * (SG[(3 * f + b) * N1 + gL] + SG[(3 * f + b) * N1 + gR]);
        float mc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) mc[t] = 0.5f * (mL[t] + mR[t]);
        float gu[4][3];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                gu[f][c] = (mc[c] * dphi[f][0] + mc[3 + c] * dphi[f][1] + mc[6 + c] * dphi[f][2]) * rjb;
        const float div3 = (gu[0][0] + gu[1][1] + gu[2][2]) * (1.0f / 3.0f);
        const float coef = SG[GF_MUEFF * N1 + gL] + SG[GF_MUEFF * N1 + gR];
        const float kap = 0.5f * (SG[GF_KAP * N1 + gL] + SG[GF_KAP * N1 + gR]);
        float tau[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            tau[i][i] = coef * (gu[i][i] - div3);
#pragma unroll
            for (int c = i + 1; c < 3; ++c) {
                tau[i][c] = coef * 0.5f * (gu[i][c] + gu[c][i]);
                tau[c][i] = tau[i][c];
            }
        }
        const float vb[3] = {0.5f * (SP[N2 + pL] + SP[N2 + pR]), 0.5f * (SP[2 * N2 + pL] + SP[2 * N2 + pR]),
                             0.5f * (SP[3 * N2 + pL] + SP[3 * N2 + pR])};
        const float *mr = mc + 3 * A;
#pragma unroll
        for (int i = 0; i < 3; ++i) H[1 + i] -= mr[0] * tau[0][i] + mr[1] * tau[1][i] + mr[2] * tau[2][i];
        float fe = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            fe += mr[c] * (tau[c][0] * vb[0] + tau[c][1] * vb[1] + tau[c][2] * vb[2] + kap * gu[3][c]);
        H[4] -= fe;
    }
}

} // namespace

template <int TY>
__global__ void __launch_bounds__(FX * TY, TY <= 8 ? 2 : 1)
    k_fused(const JetDev<float> *__restrict__ jets, const FusedJet *__restrict__ fj, int njets,
            int total_items, int src, int dst, int stage, const double *__restrict__ dt, int rhs_only)
{
    using G_ = Geo<TY>;
    extern __shared__ float S[];
    float *SP = S + G_::OFF_PRIM;
    float *SG = S + G_::OFF_GRAD;
    float *SM = S + G_::OFF_MET;
    float *SH = S + G_::OFF_HY;
    constexpr int N2 = G_::NC2, N1 = G_::NC1, C2X = G_::C2X;
    constexpr int PSLOT = NPF * N2; // floats per ring slot
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * FX + tx;
    // this thread's R1 cell is (tx, ty); its R2 cell:
    const int c2 = (ty + 1) * C2X + (tx + 1);
    const int c1 = tid;

    for (int item = blockIdx.x; item < total_items; item += gridDim.x) {
        int jet = 0;
        {
            int lo = 0, hi = njets;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (fj[mid].item0 <= item) lo = mid; else hi = mid;
            }
            jet = lo;
        }
        const JetDev<float> &J = jets[jet];
        const FusedJet &F = fj[jet];
        const FusedParams &FP = F.fp;
        int r = item - F.item0;
        const int bx = r % F.nbx;
        r /= F.nbx;
        const int by = r % F.nby;
        const int kc = r / F.nby;
        const int ni = J.n[0], nj = J.n[1], nk = J.n[2];
        const int pi = J.per[0], pj = J.per[1], pk = J.per[2];
        const int ilo = pi ? 0 : 1, ihi = pi ? ni : ni - 1;
        const int jlo = pj ? 0 : 1, jhi = pj ? nj : nj - 1;
        const int klo = pk ? 0 : 1, khi = pk ? nk : nk - 1;
        const int i0 = ilo + bx * (FX - 2), j0 = jlo + by * (TY - 2);
        const int k0 = klo + kc * F.kc;
        const int k1 = min(k0 + F.kc, khi);
        const int ib = i0 - 1, jb = j0 - 1;
        const long long fs = J.fs;
        const long long plane = (long long)nj * J.pitch;
        const float *__restrict__ Qs = J.q[src];
        const float *__restrict__ M = J.met;

        // this thread's column (R1 cell)
        const int gi = gidx(ib + tx, ni, pi), gj = gidx(jb + ty, nj, pj);
        const bool col_ok = gi >= 0 && gj >= 0;
        const long long ocol = col_ok ? (long long)gj * J.pitch + gi : 0;
        const bool out_col = tx >= 1 && tx <= FX - 2 && ty >= 1 && ty <= TY - 2 && (ib + tx) < ihi &&
                             (jb + ty) < jhi;
        const bool xi_ok = col_ok && tx <= FX - 2 && ty >= 1 && ty <= TY - 2 && (pi || gi < ni - 1);
        const bool eta_ok = col_ok && tx >= 1 && tx <= FX - 2 && ty <= TY - 2 && (pj || gj < nj - 1);
        // in-plane derivative stencils of this cell (central unless at a non-periodic end)
        const int ti = (!pi && gi == 0) ? 1 : ((!pi && gi == ni - 1) ? -1 : 0);
        const int tj = (!pj && gj == 0) ? 1 : ((!pj && gj == nj - 1) ? -1 : 0);
        // the R2 cells this thread loads in the load phase (at most two)
        int lc[2];
        long long lo2[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = tid + t * G_::NT;
            lc[t] = -1;
            lo2[t] = 0;
            if (c < N2) {
                const int ci = c % C2X, cj = c / C2X;
                const int gi2 = gidx(ib - 1 + ci, ni, pi), gj2 = gidx(jb - 1 + cj, nj, pj);
                if (gi2 >= 0 && gj2 >= 0) {
                    lc[t] = c;
                    lo2[t] = (long long)gj2 * J.pitch + gi2;
                }
            }
        }
        float hz_prev[5] = {0, 0, 0, 0, 0};
        // ring slots of planes kL-5 .. kL (sl[5] = plane kL); before the first
        // shift they describe the iteration before the first, kL = k0 - 4
        int sl[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) sl[t] = ring5(k0 - 4 - 5 + t);

        __syncthreads(); // shared memory of the previous item is free
        for (int kL = k0 - 3; kL <= k1 + 2; ++kL) {
#pragma unroll
            for (int t = 0; t < 5; ++t) sl[t] = sl[t + 1];
            sl[5] = sl[0]; // ring5(kL) == ring5(kL - 5)
            // ---- load + primitives of plane kL on R2 ----
            {
                const int gk = gidx(kL, nk, pk);
                if (gk >= 0) {
                    float *slot = SP + sl[5] * PSLOT;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (lc[t] < 0) continue;
                        const long long o = gk * plane + lo2[t];
                        const float rj = M[MET_J * fs + o];
                        const float rho = Qs[o] * rj;
                        const float rr = 1.0f / rho;
                        const float rrj = rj * rr;
                        const float u = Qs[fs + o] * rrj, v = Qs[2 * fs + o] * rrj, w = Qs[3 * fs + o] * rrj;
                        const float e = Qs[4 * fs + o] * rj;
                        const float p = FP.gm1 * (e - 0.5f * rho * (u * u + v * v + w * w));
                        const int c = lc[t];
                        slot[c] = rho;
                        slot[N2 + c] = u;
                        slot[2 * N2 + c] = v;
                        slot[3 * N2 + c] = w;
                        slot[4 * N2 + c] = p;
                        slot[5 * N2 + c] = FP.gam * p * rr;
                    }
                }
            }
            __syncthreads();
            // ---- derivatives, SGS, sensors, lambda-bar of plane kG = kL - 2 on R1 (one cell per thread) ----
            const int kG = kL - 2;
            {
                const int gk = gidx(kG, nk, pk);
                if (kG >= k0 - 1 && gk >= 0 && col_ok) {
                    float *sg = SG + ring2(kG) * NGF * N1;
                    float *sm = SM + ring2(kG) * NMF * N1;
                    const long long o = gk * plane + ocol;
                    float m[9];
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        m[t] = M[t * fs + o];
                        sm[t * N1 + c1] = m[t];
                    }
                    const float jinv = M[MET_JINV * fs + o];
                    const float csd2 = M[MET_CSD2 * fs + o];
                    sm[9 * N1 + c1] = jinv;
                    // zeta stencil of this plane (uniform): central, or one-sided at an end
                    const int tk = (!pk && gk == 0) ? 1 : ((!pk && gk == nk - 1) ? -1 : 0);
                    const float *P0 = SP + sl[3] * PSLOT; // plane kG
                    float d[4][3];
                    const int pf[4] = {1, 2, 3, 5};
                    // xi and eta derivatives from the plane-kG slot
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const int st = a == 0 ? 1 : C2X;
                        const int tt = a == 0 ? ti : tj;
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const float *Fp = P0 + pf[f] * N2 + c2;
                            float acc;
                            if (tt == 0) acc = 0.5f * (Fp[st] - Fp[-st]);
                            else if (tt > 0) acc = -1.5f * Fp[0] + 2.0f * Fp[st] - 0.5f * Fp[2 * st];
                            else acc = 1.5f * Fp[0] - 2.0f * Fp[-st] + 0.5f * Fp[-2 * st];
                            d[f][a] = acc;
                        }
                    }
                    {
                        const float *Pm2 = SP + sl[1] * PSLOT, *Pm1 = SP + sl[2] * PSLOT;
                        const float *Pp1 = SP + sl[4] * PSLOT, *Pp2 = SP + sl[5] * PSLOT;
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            const int o2 = pf[f] * N2 + c2;
                            float acc;
                            if (tk == 0) acc = 0.5f * (Pp1[o2] - Pm1[o2]);
                            else if (tk > 0) acc = -1.5f * P0[o2] + 2.0f * Pp1[o2] - 0.5f * Pp2[o2];
                            else acc = 1.5f * P0[o2] - 2.0f * Pm1[o2] + 0.5f * Pm2[o2];
                            d[f][2] = acc;
                        }
                    }
                    // pressure sensors; an end point uses its interior neighbour's
                    float nu[3];
                    {
                        const float *Pp = P0 + 4 * N2 + c2;
#pragma unroll
                        for (int a = 0; a < 2; ++a) {
                            const int st = a == 0 ? 1 : C2X;
                            const int off = (a == 0 ? ti : tj) * st;
                            const float pm = Pp[off - st], p0 = Pp[off], pp = Pp[off + st];
                            nu[a] = fabsf(pp - 2.0f * p0 + pm) / (pp + 2.0f * p0 + pm);
                        }
                        const float *Qm, *Q0, *Qp;
                        if (tk == 0) { Qm = SP + sl[2] * PSLOT; Q0 = P0; Qp = SP + sl[4] * PSLOT; }
                        else if (tk > 0) { Qm = P0; Q0 = SP + sl[4] * PSLOT; Qp = SP + sl[5] * PSLOT; }
                        else { Qm = SP + sl[1] * PSLOT; Q0 = SP + sl[2] * PSLOT; Qp = P0; }
                        const int o4 = 4 * N2 + c2;
                        const float pm = Qm[o4], p0 = Q0[o4], pp = Qp[o4];
                        nu[2] = fabsf(pp - 2.0f * p0 + pm) / (pp + 2.0f * p0 + pm);
                    }
                    const float rj = 1.0f / jinv;
                    float gu[3][3];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc)
                            gu[i][cc] = (m[cc] * d[i][0] + m[3 + cc] * d[i][1] + m[6 + cc] * d[i][2]) * rj;
                    float ss = 0.0f;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        ss += gu[i][i] * gu[i][i];
#pragma unroll
                        for (int cc = i + 1; cc < 3; ++cc) {
                            const float sic = 0.5f * (gu[i][cc] + gu[cc][i]);
                            ss += 2.0f * sic * sic;
                        }
                    }
                    const float rho = P0[c2], u = P0[N2 + c2], v = P0[2 * N2 + c2], w = P0[3 * N2 + c2],
                                T = P0[5 * N2 + c2];
                    const float mus = rho * csd2 * sqrtf(2.0f * ss);
                    const float sT = sqrtf(T);
                    const float mu = T * sT * FP.suth1 / (T + FP.suthS);
#pragma unroll
                    for (int f = 0; f < 4; ++f)
#pragma unroll
                        for (int a = 0; a < 3; ++a) sg[(3 * f + a) * N1 + c1] = d[f][a];
                    sg[GF_MUEFF * N1 + c1] = mu * FP.inv_Re + mus;
                    sg[GF_KAP * N1 + c1] = mu * FP.kap_mol + mus * FP.kap_sgs;
                    float lam[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        sg[(GF_NU + a) * N1 + c1] = nu[a];
                        const float JU = m[3 * a] * u + m[3 * a + 1] * v + m[3 * a + 2] * w;
                        const float nrm = sqrtf(m[3 * a] * m[3 * a] + m[3 * a + 1] * m[3 * a + 1] +
                                                m[3 * a + 2] * m[3 * a + 2]);
                        lam[a] = (fabsf(JU) + sT * nrm) * rj;
                    }
                    const float s01 = sqrtf(lam[0] * lam[1]), s02 = sqrtf(lam[0] * lam[2]),
                                s12 = sqrtf(lam[1] * lam[2]);
                    sg[(GF_LAM + 0) * N1 + c1] = lam[0] + s01 + s02;
                    sg[(GF_LAM + 1) * N1 + c1] = lam[1] + s01 + s12;
                    sg[(GF_LAM + 2) * N1 + c1] = lam[2] + s02 + s12;
                }
            }
            __syncthreads();
            // ---- interfaces and update of plane kU = kL - 3 ----
            const int kU = kL - 3;
            if (kU >= k0 - 1) {
                const int gk = gidx(kU, nk, pk);
                const bool plane_ok = gk >= 0;
                const int sU = sl[2] * PSLOT;
                const int g0 = ring2(kU) * NGF * N1, gm0 = ring2(kU) * NMF * N1;
                float hx[5] = {0, 0, 0, 0, 0}, hy[5] = {0, 0, 0, 0, 0}, hz[5] = {0, 0, 0, 0, 0};
                const bool first = kU == k0 - 1; // only the -1/2 zeta flux of the chunk
                if (!first && plane_ok && xi_ok) {
                    const bool lo = !pi && gi == 0, hi = !pi && gi + 1 == ni - 1;
                    fused_iface<0, TY>(S, FP, sU + c2 - 1, sU + c2, sU + c2 + 1, sU + c2 + 2, g0 + c1, g0 + c1 + 1,
                                       gm0 + c1, gm0 + c1 + 1, lo, hi, hx);
                }
                if (!first && plane_ok && eta_ok) {
                    const bool lo = !pj && gj == 0, hi = !pj && gj + 1 == nj - 1;
                    fused_iface<1, TY>(S, FP, sU + c2 - C2X, sU + c2, sU + c2 + C2X, sU + c2 + 2 * C2X, g0 + c1,
                                       g0 + c1 + FX, gm0 + c1, gm0 + c1 + FX, lo, hi, hy);
                }
                if (plane_ok && out_col && (pk || gk < nk - 1)) {
                    const bool lo = !pk && gk == 0, hi = !pk && gk + 1 == nk - 1;
                    fused_iface<2, TY>(S, FP, sl[1] * PSLOT + c2, sU + c2, sl[3] * PSLOT + c2, sl[4] * PSLOT + c2,
                                       g0 + c1, ring2(kU + 1) * NGF * N1 + c1, gm0 + c1,
                                       ring2(kU + 1) * NMF * N1 + c1, lo, hi, hz);
                }
                float hxm[5];
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    hxm[f] = __shfl_up_sync(0xffffffffu, hx[f], 1);
                    SH[(f * TY + ty) * FX + tx] = hy[f];
                }
                __syncthreads();
                if (!first && plane_ok && out_col && kU < k1) {
                    const long long o = gk * plane + ocol;
                    float R[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f)
                        R[f] = (hx[f] - hxm[f]) + (hy[f] - SH[(f * TY + ty - 1) * FX + tx]) + (hz[f] - hz_prev[f]);
                    if (rhs_only) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) J.rhs[f * fs + o] = R[f];
                    } else {
                        const float adt = c_alpha_f[stage] * (float)dt[jet];
                        const float *Q0 = J.q[0];
                        float *Qd = J.q[dst];
#pragma unroll
                        for (int f = 0; f < 5; ++f) Qd[f * fs + o] = Q0[f * fs + o] - adt * R[f];
                    }
                }
#pragma unroll
                for (int f = 0; f < 5; ++f) hz_prev[f] = hz[f];
            }
            __syncthreads();
        }
    }
}

template <int TY> size_t fused_smem_bytes() { return Geo<TY>::BYTES; }

template <int TY> int fused_prepare()
{
    return (int)cudaFuncSetAttribute(k_fused<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Geo<TY>::BYTES);
}

template <int TY>
void launch_fused(const JetDev<float> *jets, const FusedJet *fj, int njets, int total_items, int grid, int src,
                  int dst, int stage, const double *dt, int rhs_only, cudaStream_t st)
{
    dim3 block(FX, TY);
    k_fused<TY><<<grid, block, Geo<TY>::BYTES, st>>>(jets, fj, njets, total_items, src, dst, stage, dt,
                                                    rhs_only);
}

template size_t fused_smem_bytes<16>();
template size_t fused_smem_bytes<8>();
template int fused_prepare<16>();
template int fused_prepare<8>();
template void launch_fused<16>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int,
                               const double *, int, cudaStream_t);
template void launch_fused<8>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int,
                              const double *, int, cudaStream_t);

} // namespace les
