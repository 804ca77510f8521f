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
// in registers while marching along k).  All three have this thread's point
// on their low side, so its data are read from shared memory once per plane.
// Point data live in a ring of 5 planes over R2 = R1 plus one column/row on
// each side, so that derivatives — one-sided at a non-periodic end included —
// of plane k are formed when plane k+2 arrives; derivatives, transport
// coefficients, sensors, lambda-bar and metrics of R1 are kept for two
// planes.  Shared memory holds cells as float4/float2 records so that one
// vector load fetches a point's primitives, derivatives or metric row
// (the stage is issue-bound, and this cuts load instructions about 3x).
// Per loaded plane kL:  load+primitives(kL), metrics(kL-2) | gradients(kL-2)
// | interfaces+update(kL-3).  The 32 x 8 variant fits two CTAs per SM, so the
// load phase of one overlaps the arithmetic of the other.
//
// Work list.  Items (jet, tile x, tile y, k-chunk) are walked by a persistent
// grid in a fixed order; results do not depend on the item order, the chunk
// length or the grid size.
#include <cmath>

#include "les_internal.cuh"

namespace les {

namespace {

constexpr int FX = 32; // threads along i (one warp per row)

__constant__ float c_alpha_f[5] = {0.25f, 1.0f / 6.0f, 0.375f, 0.5f, 1.0f};

// Shared-memory map (byte offsets).  float4 records first (16-byte aligned).
//   PA [5][NC2] float4  rho u v w       (point ring)
//   GD [2][3][NC1] float4  d(u,v,w,T)/d xi_a, a = 0..2
//   GC [2][2][NC1] float4  (mu_eff, kappa, nu_xi, lb_xi), (nu_eta, lb_eta, nu_zeta, lb_zeta)
//   MA [2][2][NC1] float4  metric cofactors m0..m3, m4..m7
//   MB [2][NC1] float2  m8, J^-1
//   PB [5][NC2] float2  p T              (point ring)
//   SH [5][TY][FX] float  eta-interface fluxes of the current plane
//   HX [C2X], HY [C2Y] float4  separable form: (h, 1/h, h^(2/3), 0) of the
//                              tile's columns / rows, h = dx/dxi resp. dy/deta
//   QG [5][C2Y][40] float       general form (in place of HX, HY, 128-byte
//                              aligned): the next plane's state box, staged
//                              by one TMA copy; then its mbarrier (8 bytes)
template <int TY> struct Geo {
    static constexpr int NT = FX * TY;
    static constexpr int C2X = FX + 2, C2Y = TY + 2, NC2 = C2X * C2Y; // R2: cells [-1, FX] x [-1, TY]
    static constexpr int NC1 = FX * TY;                                // R1: the thread grid
    static constexpr size_t O_PA = 0;
    static constexpr size_t O_GD = O_PA + 16ull * 5 * NC2;
    static constexpr size_t O_GC = O_GD + 16ull * 2 * 3 * NC1;
    static constexpr size_t O_MA = O_GC + 16ull * 2 * 2 * NC1;
    static constexpr size_t O_MB = O_MA + 16ull * 2 * 2 * NC1;
    static constexpr size_t O_PB = O_MB + 8ull * 2 * NC1;
    static constexpr size_t O_SH = O_PB + 8ull * 5 * NC2;
    // separable form: MA/MB hold no metrics; 10 NT floats of them stage the
    // state of the next plane (cp.async), see k_fused
    static constexpr size_t O_QS = O_MA; // float [2 cells][5][NT]
    static_assert(O_QS + 4ull * 10 * NT <= O_PB, "staging fits in MA+MB");
    static constexpr size_t O_HX = O_SH + 4ull * 5 * TY * FX;
    static constexpr size_t O_HY = O_HX + 16ull * C2X;
    static constexpr size_t BYTES_SEP = O_HY + 16ull * C2Y;
    static constexpr unsigned BOX_BYTES = 4u * 5 * C2Y * TMA_BOX_X;
    static_assert(BOX_BYTES % 16 == 0, "box size");
    // TMA box and its mbarrier: after the eta-flux rows (general form), or
    // in the metric-table region the separable form does not use
    static constexpr size_t O_QG = (O_HX + 127) / 128 * 128;
    static constexpr size_t O_MBAR = O_QG + BOX_BYTES;
    static constexpr size_t BYTES_GEN = O_MBAR + 8;
    static constexpr size_t O_QG_SEP = (O_MA + 127) / 128 * 128;
    static constexpr size_t O_MBAR_SEP = O_QG_SEP + BOX_BYTES;
    static_assert(O_MBAR_SEP + 8 <= O_PB, "separable form: box fits in the metric-table region");
    static constexpr size_t bytes(bool sep) { return sep ? BYTES_SEP : BYTES_GEN; }
};

template <int TY> struct Sm {
    float4 *PA, *GD, *GC, *MA;
    float2 *PB, *MB;
    float *SH;
    float4 *HX, *HY;
    float *QS, *QG;
    unsigned long long *MBAR;
    __device__ __forceinline__ Sm(unsigned char *b, bool sep)
        : PA((float4 *)(b + Geo<TY>::O_PA)), GD((float4 *)(b + Geo<TY>::O_GD)),
          GC((float4 *)(b + Geo<TY>::O_GC)), MA((float4 *)(b + Geo<TY>::O_MA)),
          PB((float2 *)(b + Geo<TY>::O_PB)), MB((float2 *)(b + Geo<TY>::O_MB)), SH((float *)(b + Geo<TY>::O_SH)),
          HX((float4 *)(b + Geo<TY>::O_HX)), HY((float4 *)(b + Geo<TY>::O_HY)),
          QS((float *)(b + Geo<TY>::O_QS)), QG((float *)(b + (sep ? Geo<TY>::O_QG_SEP : Geo<TY>::O_QG))),
          MBAR((unsigned long long *)(b + (sep ? Geo<TY>::O_MBAR_SEP : Geo<TY>::O_MBAR)))
    {
    }
};

__device__ __forceinline__ int ring5(int k) { return ((k % 5) + 5) % 5; }
__device__ __forceinline__ int ring2(int k) { return k & 1; } // two's complement: -1 -> 1

// Wrap a global index on a periodic axis; -1 for outside a non-periodic axis.
__device__ __forceinline__ int gidx(int g, int n, int per)
{
    if (per) {
        // the tile and plane indices stray at most one period: a compare and
        // an add, with the modulo only as a fallback
        const int h = g < 0 ? g + n : (g >= n ? g - n : g);
        return (unsigned)h < (unsigned)n ? h : wrapi(g, n);
    }
    return (g >= 0 && g < n) ? g : -1;
}

// Square root of a strictly positive argument through the hardware
// reciprocal square root (max. 2 ulp): x * rsqrt(x).
__device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }
// The same for x >= 0 (0 -> 0): a spectral radius vanishes on the axis of a
// polar mesh, so the products of lambda-bar can be zero.
__device__ __forceinline__ float sqrt_nonneg(float x) { return x * rsqrtf(fmaxf(x, 1.17549435e-38f)); }

// Asynchronous 4-byte global -> shared copy (completes without the issuing
// thread waiting; cp_async_wait_all() waits for all of this thread's copies).
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// TMA staging of the general form: an mbarrier with one arrival (the issuing
// thread's, carrying the expected byte count) completed by the copy.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); // visible to the copy engine
}
// 4-D tiled copy (x, y, z, field) of the tensor map's box into shared memory;
// x must be a multiple of 4 elements (16 bytes); other coordinates may lie
// outside the tensor (zero fill).
__device__ __forceinline__ void tma_box_load(float *dst, const CUtensorMap *map, int x, int y, int z,
                                             unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(bar))
                 : "memory");
}
// Wait for the phase of the given parity, polling at most `limit` times
// (false: gave up).
constexpr int MBAR_WAIT_LIMIT = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}


__device__ __forceinline__ float cmp(const float4 &v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Dissipation vector W = [rho, rho u, rho v, rho w, e + p] of a point.
__device__ __forceinline__ void wvec(const float4 &a, float p, float hg, float W[5])
{
    W[0] = a.x;
    W[1] = a.x * a.y;
    W[2] = a.x * a.z;
    W[3] = a.x * a.w;
    W[4] = hg * p + 0.5f * a.x * (a.y * a.y + a.z * a.z + a.w * a.w);
}

// Data of the thread's own point at the interface plane; it is the low
// side (L) of all three interfaces the thread evaluates.
struct OwnPt {
    float4 a; // rho u v w
    float p, T;
    float m[9], jinv;
    int c1, pl; // R1 cell and R1 plane (ring2) of the point
};

// Flux through the interface between the own point L and its +A neighbour R
// (Eqs. spatial_discret, inv_flux_vec, dissip_term; compact viscous flux of
// the interface).  Shared-memory indices: r2/lm2/rp2 of R, L-1 and R+1 in
// the point ring; r1 of R in the R1 tables, rpl the R1 plane (ring2) of R.
template <int A, int TY>
__device__ __forceinline__ void fused_iface(const Sm<TY> &S, const FusedParams &FP, const OwnPt &L, int r2,
                                            int lm2, int rp2, int r1, int rpl, bool lo_end, bool hi_end,
                                            float H[5])
{
    constexpr int N1 = Geo<TY>::NC1;
    const float hg = FP.hgam;
    float LW[5];
    wvec(L.a, L.p, hg, LW);
    // R point and the two outer points of the dissipation stencil
    const float4 ra = S.PA[r2];
    const float2 rb = S.PB[r2];
    float WR[5], WLm[5], WRp[5];
    wvec(ra, rb.x, hg, WR);
    if (!lo_end) {
        const float4 q = S.PA[lm2];
        wvec(q, S.PB[lm2].x, hg, WLm);
    }
    if (!hi_end) {
        const float4 q = S.PA[rp2];
        wvec(q, S.PB[rp2].x, hg, WRp);
    }
    // metric rows at R
    float mR[9];
    const float4 u0 = S.MA[(rpl * 2 + 0) * N1 + r1], u1 = S.MA[(rpl * 2 + 1) * N1 + r1];
    const float2 u2 = S.MB[rpl * N1 + r1];
    mR[0] = u0.x; mR[1] = u0.y; mR[2] = u0.z; mR[3] = u0.w;
    mR[4] = u1.x; mR[5] = u1.y; mR[6] = u1.z; mR[7] = u1.w;
    mR[8] = u2.x;
    const float jb = 0.5f * (L.jinv + u2.y);
    // centred inviscid flux 0.5 (F_L + F_R), J^-1 U = m_A . u
    {
        const float JUL = L.m[3 * A] * L.a.y + L.m[3 * A + 1] * L.a.z + L.m[3 * A + 2] * L.a.w;
        const float JUR = mR[3 * A] * ra.y + mR[3 * A + 1] * ra.z + mR[3 * A + 2] * ra.w;
        H[0] = 0.5f * (LW[0] * JUL + WR[0] * JUR);
        // pressure terms with the ambient pressure taken out: a constant
        // pressure has no flux divergence (metric identities), and leaving it
        // in would add FP32 rounding of O(1) terms to the small transverse
        // momentum residuals, and the metric identities' FP32 round-off
        // times p_inf as a spurious source
        const float pL = L.p - FP.pinf, pR = rb.x - FP.pinf;
        H[1] = 0.5f * (LW[1] * JUL + pL * L.m[3 * A] + WR[1] * JUR + pR * mR[3 * A]);
        H[2] = 0.5f * (LW[2] * JUL + pL * L.m[3 * A + 1] + WR[2] * JUR + pR * mR[3 * A + 1]);
        H[3] = 0.5f * (LW[3] * JUL + pL * L.m[3 * A + 2] + WR[3] * JUR + pR * mR[3 * A + 2]);
        H[4] = 0.5f * (LW[4] * JUL + WR[4] * JUR);
    }
    // transport coefficients, sensor and lambda-bar at R
    float mueR, kapR, nuR, lbR;
    if (A == 0) {
        const float4 c = S.GC[(rpl * 2 + 0) * N1 + r1];
        mueR = c.x; kapR = c.y; nuR = c.z; lbR = c.w;
    } else {
        const float2 c = *reinterpret_cast<const float2 *>(&S.GC[(rpl * 2 + 0) * N1 + r1]);
        const float2 e = reinterpret_cast<const float2 *>(&S.GC[(rpl * 2 + 1) * N1 + r1])[A - 1];
        mueR = c.x; kapR = c.y; nuR = e.x; lbR = e.y;
    }
    float mueL, kapL, nuL, lbL;
    if (A == 0) {
        const float4 c = S.GC[(L.pl * 2 + 0) * N1 + L.c1];
        mueL = c.x; kapL = c.y; nuL = c.z; lbL = c.w;
    } else {
        const float2 c = *reinterpret_cast<const float2 *>(&S.GC[(L.pl * 2 + 0) * N1 + L.c1]);
        const float2 e = reinterpret_cast<const float2 *>(&S.GC[(L.pl * 2 + 1) * N1 + L.c1])[A - 1];
        mueL = c.x; kapL = c.y; nuL = e.x; lbL = e.y;
    }
    // Turkel-Vatsa dissipation
    {
        const float eps2 = FP.k2 * fmaxf(nuL, nuR);
        const float eps4 = fmaxf(0.0f, FP.k4 - eps2);
        const float sc = jb * 0.5f * (lbL + lbR);
        const float se2 = sc * eps2, se4 = sc * eps4;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            // dW(+3/2) - 2 dW(+1/2) + dW(-1/2) = W(R+1) - W(L-1) - 3 dW(+1/2); at a
            // non-periodic end the mirrored difference makes W(R+1) = W(L), W(L-1) = W(R)
            const float dW0 = WR[f] - LW[f];
            const float d3 = ((hi_end ? LW[f] : WRp[f]) - (lo_end ? WR[f] : WLm[f])) - 3.0f * dW0;
            H[f] += se4 * d3 - se2 * dW0;
        }
    }
    // compact viscous + SGS flux
    {
        const float rjb = __fdividef(1.0f, jb);
        constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2; // tangential axes
        const float4 dR1 = S.GD[(rpl * 3 + B1) * N1 + r1], dR2 = S.GD[(rpl * 3 + B2) * N1 + r1];
        const float4 dL1 = S.GD[(L.pl * 3 + B1) * N1 + L.c1], dL2 = S.GD[(L.pl * 3 + B2) * N1 + L.c1];
        float dphi[4][3];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float lv = f == 0 ? L.a.y : (f == 1 ? L.a.z : (f == 2 ? L.a.w : L.T));
            const float rv = f == 0 ? ra.y : (f == 1 ? ra.z : (f == 2 ? ra.w : rb.y));
            dphi[f][A] = rv - lv;
            dphi[f][B1] = 0.5f * (cmp(dL1, f) + cmp(dR1, f));
            dphi[f][B2] = 0.5f * (cmp(dL2, f) + cmp(dR2, f));
        }
        float mc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) mc[t] = 0.5f * (L.m[t] + mR[t]);
        float gu[4][3];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                gu[f][c] = (mc[c] * dphi[f][0] + mc[3 + c] * dphi[f][1] + mc[6 + c] * dphi[f][2]) * rjb;
        const float div3 = (gu[0][0] + gu[1][1] + gu[2][2]) * (1.0f / 3.0f);
        const float coef = mueL + mueR;
        const float kap = 0.5f * (kapL + kapR);
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
        const float vb[3] = {0.5f * (L.a.y + ra.y), 0.5f * (L.a.z + ra.z), 0.5f * (L.a.w + ra.w)};
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

// Separable form of fused_iface on a Cartesian-product grid x = x(i),
// y = y(j), z = z(k) (Sec. "Transformation of Coordinates" with diagonal
// metrics): the cofactor matrix is diag(y_eta z_zeta, x_xi z_zeta,
// x_xi y_eta), so the face factor of axis A is the product Sa of the two
// tangential spacings (equal on both sides), J^-1 at the interface is
// Sa * hb with hb the interface average of the spacing along A, and the
// chain rule reduces to d/dx_c = (1/h_c) d/dxi_c.  hAL, hAR: spacing along A
// at L and R; hT1/rhT1, hT2/rhT2: the tangential spacings and reciprocals
// (axes B1 < B2).
template <int A, int TY>
__device__ __forceinline__ void fused_iface_sep(const Sm<TY> &S, const FusedParams &FP, const OwnPt &L, int r2,
                                                int lm2, int rp2, int r1, int rpl, bool lo_end, bool hi_end,
                                                float hAL, float hAR, float hT1, float rhT1, float hT2,
                                                float rhT2, float H[5])
{
    constexpr int N1 = Geo<TY>::NC1;
    const float hg = FP.hgam;
    float LW[5];
    wvec(L.a, L.p, hg, LW);
    const float4 ra = S.PA[r2];
    const float2 rb = S.PB[r2];
    float WR[5], WLm[5], WRp[5];
    wvec(ra, rb.x, hg, WR);
    if (!lo_end) {
        const float4 q = S.PA[lm2];
        wvec(q, S.PB[lm2].x, hg, WLm);
    }
    if (!hi_end) {
        const float4 q = S.PA[rp2];
        wvec(q, S.PB[rp2].x, hg, WRp);
    }
    const float Sa = hT1 * hT2;
    const float hb = 0.5f * (hAL + hAR);
    const float jb = Sa * hb;
    // centred inviscid flux: J^-1 U_A = Sa u_A on both sides
    {
        const float JUL = Sa * cmp(L.a, 1 + A), JUR = Sa * cmp(ra, 1 + A);
#pragma unroll
        for (int f = 0; f < 5; ++f) H[f] = 0.5f * (LW[f] * JUL + WR[f] * JUR);
        H[1 + A] += 0.5f * Sa * ((L.p - FP.pinf) + (rb.x - FP.pinf)); // ambient pressure out, as above
    }
    float mueL, kapL, nuL, lbL, mueR, kapR, nuR, lbR;
    if (A == 0) {
        const float4 c = S.GC[(L.pl * 2 + 0) * N1 + L.c1], d = S.GC[(rpl * 2 + 0) * N1 + r1];
        mueL = c.x; kapL = c.y; nuL = c.z; lbL = c.w;
        mueR = d.x; kapR = d.y; nuR = d.z; lbR = d.w;
    } else {
        const float2 c = *reinterpret_cast<const float2 *>(&S.GC[(L.pl * 2 + 0) * N1 + L.c1]);
        const float2 e = reinterpret_cast<const float2 *>(&S.GC[(L.pl * 2 + 1) * N1 + L.c1])[A - 1];
        const float2 d = *reinterpret_cast<const float2 *>(&S.GC[(rpl * 2 + 0) * N1 + r1]);
        const float2 g = reinterpret_cast<const float2 *>(&S.GC[(rpl * 2 + 1) * N1 + r1])[A - 1];
        mueL = c.x; kapL = c.y; nuL = e.x; lbL = e.y;
        mueR = d.x; kapR = d.y; nuR = g.x; lbR = g.y;
    }
    // Turkel-Vatsa dissipation
    {
        const float eps2 = FP.k2 * fmaxf(nuL, nuR);
        const float eps4 = fmaxf(0.0f, FP.k4 - eps2);
        const float sc = jb * 0.5f * (lbL + lbR);
        const float se2 = sc * eps2, se4 = sc * eps4;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            // dW(+3/2) - 2 dW(+1/2) + dW(-1/2) = W(R+1) - W(L-1) - 3 dW(+1/2); at a
            // non-periodic end the mirrored difference makes W(R+1) = W(L), W(L-1) = W(R)
            const float dW0 = WR[f] - LW[f];
            const float d3 = ((hi_end ? LW[f] : WRp[f]) - (lo_end ? WR[f] : WLm[f])) - 3.0f * dW0;
            H[f] += se4 * d3 - se2 * dW0;
        }
    }
    // compact viscous + SGS flux: only row A of the stress tensor is needed
    {
        const float rhb = __fdividef(1.0f, hb);
        constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
        const float4 dR1 = S.GD[(rpl * 3 + B1) * N1 + r1], dR2 = S.GD[(rpl * 3 + B2) * N1 + r1];
        const float4 dL1 = S.GD[(L.pl * 3 + B1) * N1 + L.c1], dL2 = S.GD[(L.pl * 3 + B2) * N1 + L.c1];
        float gu[4][3];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float lv = f == 0 ? L.a.y : (f == 1 ? L.a.z : (f == 2 ? L.a.w : L.T));
            const float rv = f == 0 ? ra.y : (f == 1 ? ra.z : (f == 2 ? ra.w : rb.y));
            gu[f][A] = (rv - lv) * rhb;
            gu[f][B1] = 0.5f * (cmp(dL1, f) + cmp(dR1, f)) * rhT1;
            gu[f][B2] = 0.5f * (cmp(dL2, f) + cmp(dR2, f)) * rhT2;
        }
        const float div3 = (gu[0][0] + gu[1][1] + gu[2][2]) * (1.0f / 3.0f);
        const float coef = mueL + mueR;
        const float kap = 0.5f * (kapL + kapR);
        float tA[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) tA[i] = i == A ? coef * (gu[A][A] - div3) : coef * 0.5f * (gu[A][i] + gu[i][A]);
        const float vb0 = 0.5f * (L.a.y + ra.y), vb1 = 0.5f * (L.a.z + ra.z), vb2 = 0.5f * (L.a.w + ra.w);
#pragma unroll
        for (int i = 0; i < 3; ++i) H[1 + i] -= Sa * tA[i];
        H[4] -= Sa * (tA[0] * vb0 + tA[1] * vb1 + tA[2] * vb2 + kap * gu[3][A]);
    }
}

// Derivative along one axis of (u, v, w, T) and the pressure sensor of the
// point at ring offset 0, from the points at offsets -s, 0, +s (central) or,
// at a non-periodic end, the one-sided second-order stencil (the sensor of
// an end point is its interior neighbour's: same three points).
struct D3 {
    float4 d;
    float nu;
};

__device__ __forceinline__ D3 deriv_central(const float4 &am, const float2 &bm, float p0, const float4 &ap,
                                            const float2 &bp)
{
    D3 r;
    r.d = make_float4(0.5f * (ap.y - am.y), 0.5f * (ap.z - am.z), 0.5f * (ap.w - am.w), 0.5f * (bp.y - bm.y));
    r.nu = __fdividef(fabsf(bp.x - 2.0f * p0 + bm.x), bp.x + 2.0f * p0 + bm.x);
    return r;
}

// Points q1, q2, q3 at offsets (t-1, t, t+1) s, t = +1 (start) or -1 (end).
__device__ __forceinline__ D3 deriv_end(int t, const float4 &a1, const float2 &b1, const float4 &a2,
                                        const float2 &b2, const float4 &a3, const float2 &b3)
{
    // forward  (t = +1): -1.5 q(0) + 2 q(s) - 0.5 q(2s)  = -1.5 q1 + 2 q2 - 0.5 q3
    // backward (t = -1):  1.5 q(0) - 2 q(-s) + 0.5 q(-2s) = 0.5 q1 - 2 q2 + 1.5 q3
    const float c1 = t > 0 ? -1.5f : 0.5f, c2 = t > 0 ? 2.0f : -2.0f, c3 = t > 0 ? -0.5f : 1.5f;
    D3 r;
    r.d = make_float4(c1 * a1.y + c2 * a2.y + c3 * a3.y, c1 * a1.z + c2 * a2.z + c3 * a3.z,
                      c1 * a1.w + c2 * a2.w + c3 * a3.w, c1 * b1.y + c2 * b2.y + c3 * b3.y);
    r.nu = __fdividef(fabsf(b3.x - 2.0f * b2.x + b1.x), b3.x + 2.0f * b2.x + b1.x);
    return r;
}

} // namespace

// Index checks of a LES_BOUNDS_CHECK build (nothing otherwise): global
// offsets against the padded point count, shared-memory slots against their
// tables (point ring 5 NC2 cells, plane tables 2 x (3 or 2) NC1 cells,
// eta-flux rows 5 TY FX).
#define CK_G(site, x) LES_BOUNDS(J.oob, (site), (x), J.npts_pad)
#define CK_RING(x) ((int)LES_BOUNDS(J.oob, 5, (x), 5 * N2))
#define CK_TAB(x, n) ((int)LES_BOUNDS(J.oob, 6, (x), (n)))
#define CK_SH(x) ((int)LES_BOUNDS(J.oob, 7, (x), 5 * TY * FX))

template <int TY, bool SEP>
__global__ void __launch_bounds__(FX * TY, TY <= 8 ? 2 : 1)
    k_fused(const JetDev<float> *__restrict__ jets, const FusedJet *__restrict__ fj, int njets,
            int total_items, int total_tiles, int src, int dst, int stage, const double *__restrict__ dt,
            int rhs_only, int balanced, int wait_limit)
{
    using G_ = Geo<TY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Sm<TY> S(smem_raw, SEP);
    constexpr int N2 = G_::NC2, N1 = G_::NC1, C2X = G_::C2X;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * FX + tx;
    // this thread's R1 cell is (tx, ty); its R2 cell:
    const int c2 = (ty + 1) * C2X + (tx + 1);
    const int c1 = tid;

    // Work cursor: items (jet, tile, k-chunk) strided over the grid
    // (balanced = 0), or the CTA's contiguous, equal share of all tile-planes
    // (jet-major, tile, then plane), cut into one column piece per tile it
    // touches (balanced = 1).  balanced = 2 (lockstep) first runs
    // total_tiles / gridDim.x waves of whole columns (tile blockIdx.x +
    // wave * gridDim.x: the CTAs march k together, so neighbouring tiles read
    // their shared halo planes within a short window, mostly from L2) and
    // shares out the remaining tile-planes the same way.  A piece starting
    // mid-column recomputes its first zeta flux, so the result does not
    // depend on where the cuts fall.
    // general form: the TMA staging buffer must be 128-byte aligned (the
    // dynamic shared memory starts the window, so it is; checked anyway)
    const bool tma_smem_ok = (smem_u32(S.QG) & 127u) == 0;
    unsigned tpar = 0; // parity of the next staging phase
    // A staging wait that gives up (wait_limit polls) is recorded in the
    // jet's error word (site 8); from the next barrier on the whole CTA reads
    // the state directly from global memory for the rest of the launch, and
    // thread 0, which issued the outstanding copy, waits for it (bounded)
    // before the CTA exits.
    bool tma_off = false, pend = false;
    if (tid == 0) mbar_init(S.MBAR);
    __syncthreads();
    int item = blockIdx.x, w = 0, wend = 0;
    // balanced form: tile-plane ranges [w, wend), one per whole-column wave,
    // then the share of the rest
    const int nwave = balanced == 2 ? total_tiles / (int)gridDim.x : 0;
    int wave = 0;
    auto jet_of_tile = [&](int t) {
        int lo = 0, hi = njets;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (fj[mid].tile0 <= t) lo = mid; else hi = mid;
        }
        return lo;
    };
    auto next_range = [&]() {
        while (wave <= nwave) {
            if (wave < nwave) {
                const int t = blockIdx.x + wave * gridDim.x;
                const FusedJet &Fw = fj[jet_of_tile(t)];
                w = Fw.item0 + (t - Fw.tile0) * Fw.nkc;
                wend = w + Fw.nkc;
            } else {
                const int t1 = nwave * gridDim.x;
                int i1 = total_items;
                if (t1 < total_tiles) {
                    const FusedJet &Fw = fj[jet_of_tile(t1)];
                    i1 = Fw.item0 + (t1 - Fw.tile0) * Fw.nkc;
                }
                const long long rem = total_items - i1;
                w = i1 + (int)((rem * blockIdx.x) / gridDim.x);
                wend = i1 + (int)((rem * (blockIdx.x + 1)) / gridDim.x);
            }
            ++wave;
            if (w < wend) return true;
        }
        return false;
    };
    if (balanced) next_range();
    while (balanced ? (w < wend || next_range()) : item < total_items) {
        const int key = balanced ? w : item;
        int jet = 0;
        {
            int lo = 0, hi = njets;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (fj[mid].item0 <= key) lo = mid; else hi = mid;
            }
            jet = lo;
        }
        const JetDev<float> &J = jets[jet];
        const FusedJet &F = fj[jet];
        const FusedParams &FP = F.fp;
        const int ni = J.n[0], nj = J.n[1], nk = J.n[2];
        const int pi = J.per[0], pj = J.per[1], pk = J.per[2];
        const int ilo = pi ? 0 : 1, ihi = pi ? ni : ni - 1;
        const int jlo = pj ? 0 : 1, jhi = pj ? nj : nj - 1;
        const int klo = pk ? 0 : 1, khi = pk ? nk : nk - 1;
        int bx, by, k0, k1;
        if (balanced) {
            const int np = khi - klo; // planes per column (F.nkc)
            const int r = key - F.item0;
            const int tile = r / np, pl = r - tile * np;
            bx = tile % F.nbx;
            by = tile / F.nbx;
            k0 = klo + pl;
            k1 = klo + min(np, pl + (wend - w));
            w += k1 - k0;
        } else {
            int r = key - F.item0;
            bx = r % F.nbx;
            r /= F.nbx;
            by = r % F.nby;
            const int kc = r / F.nby;
            k0 = klo + kc * F.kc;
            k1 = min(k0 + F.kc, khi);
            item += gridDim.x;
        }
        const int i0 = ilo + bx * (FX - 2), j0 = jlo + by * (TY - 2);
        const int ib = i0 - 1, jb = j0 - 1;
        const long long fs = J.fs;
        const long long plane = (long long)nj * J.pitch;
        const float *__restrict__ Qs = J.q[src];
        float *__restrict__ Qd = J.q[dst];
        const float adt = rhs_only ? 0.0f : c_alpha_f[stage] * (float)dt[jet];

        // this thread's column (R1 cell)
        const int gi = gidx(ib + tx, ni, pi), gj = gidx(jb + ty, nj, pj);
        const bool col_ok = gi >= 0 && gj >= 0;
        const long long ocol = col_ok ? (long long)gj * J.pitch + gi : 0;
        const bool out_col = tx >= 1 && tx <= FX - 2 && ty >= 1 && ty <= TY - 2 && (ib + tx) < ihi &&
                             (jb + ty) < jhi;
        const bool xi_ok = col_ok && tx <= FX - 2 && ty >= 1 && ty <= TY - 2 && (pi || gi < ni - 1);
        const bool eta_ok = col_ok && tx >= 1 && tx <= FX - 2 && ty <= TY - 2 && (pj || gj < nj - 1);
        const bool xi_lo = !pi && gi == 0, xi_hi = !pi && gi + 1 == ni - 1;
        const bool eta_lo = !pj && gj == 0, eta_hi = !pj && gj + 1 == nj - 1;
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
        // jets with no periodic i or j axis: the plane's state arrives as one
        // TMA box [5][C2Y][40] whose x starts at the tile's first column
        // rounded down to a multiple of 4; qg[t] is load cell t's offset in it
        const CUtensorMap *tmap = nullptr;
        int qg[2] = {0, 0}, tx0 = 0;
        if (F.tmap && tma_smem_ok && !pi && !pj && !tma_off) {
            tmap = F.tmap + (TY == 16 ? 3 : 0) + src;
            tx0 = (ib - 1) & ~3;
#pragma unroll
            for (int t = 0; t < 2; ++t)
                if (lc[t] >= 0) qg[t] = (lc[t] / C2X) * TMA_BOX_X + (ib - 1 - tx0) + lc[t] % C2X;
        }
        if constexpr (SEP) {
            // 1-D spacings of the tile's columns and rows (the previous item's
            // last reads of HX/HY precede its closing barrier)
            if (tid < C2X) {
                const int g = gidx(ib - 1 + tid, ni, pi);
                S.HX[tid] = g >= 0 ? F.h1[0][g] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            } else if (tid < C2X + G_::C2Y) {
                const int t = tid - C2X;
                const int g = gidx(jb - 1 + t, nj, pj);
                S.HY[t] = g >= 0 ? F.h1[1][g] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        float hz_prev[5] = {0, 0, 0, 0, 0};
        // ring slots of planes kL-5 .. kL (sl[5] = plane kL); before the first
        // shift they describe the iteration before the first, kL = k0 - 4
        int sl[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) sl[t] = ring5(k0 - 4 - 5 + t);

        // J of this thread's column at the plane of the next update (the
        // state is stored unscaled, so the update is Q(l) = Q(0) - alpha dt J R)
        float rjU = 0.0f;
        __syncthreads(); // shared memory of the previous item is free
        // separable form without a tensor map: the state of plane kq at this
        // thread's load cells is staged in shared memory one iteration ahead by
        // asynchronous copies, so the load phase finds it there; each thread
        // reads only what it copied
        auto stage_q = [&](int kq) {
            const int gk = gidx(kq, nk, pk);
            if (kq > k1 + 2 || gk < 0) return;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (lc[t] < 0) continue;
                const long long o = CK_G(2, gk * plane + lo2[t]);
#pragma unroll
                for (int f = 0; f < 5; ++f) cp_async4(&S.QS[(t * 5 + f) * G_::NT + tid], Qs + f * fs + o);
            }
        };
        // with a tensor map: thread 0 issues the box of plane kq once every
        // thread is done with the previous one (after a barrier)
        auto stage_box = [&](int kq) {
            const int gk = gidx(kq, nk, pk);
            if (kq > k1 + 2 || gk < 0 || tid != 0) return;
            tma_box_load(S.QG, tmap, tx0, jb - 1, gk, S.MBAR, G_::BOX_BYTES);
        };
        if (tmap) {
            stage_box(k0 - 3);
        } else if (SEP && !tma_off) {
            stage_q(k0 - 3);
            cp_async_commit();
        }
        for (int kL = k0 - 3; kL <= k1 + 2; ++kL) {
#pragma unroll
            for (int t = 0; t < 5; ++t) sl[t] = sl[t + 1];
            sl[5] = sl[0]; // ring5(kL) == ring5(kL - 5)
            const int kG = kL - 2;
            const int gkG = gidx(kG, nk, pk);
            const bool g_act = kG >= k0 - 1 && gkG >= 0 && col_ok;
            const int rG = ring2(kG);
            // ---- static fields of plane kG (R1, this thread's column) and
            //      load + primitives of plane kL on R2; every global load of
            //      the phase is issued before the first shared-memory store,
            //      so that their latencies overlap ----
            float m[9], jinvG = 0.0f, csd2 = 0.0f, rjG = 0.0f, nrm[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int t = 0; t < 9; ++t) m[t] = 0.0f;
            if (!SEP && g_act) {
                const float4 *mp = F.mp + 4 * CK_G(3, gkG * plane + ocol);
                const float4 a0 = mp[0], a1 = mp[1], a2 = mp[2], a3 = mp[3];
                m[0] = a0.x; m[1] = a0.y; m[2] = a0.z; m[3] = a0.w;
                m[4] = a1.x; m[5] = a1.y; m[6] = a1.z; m[7] = a1.w;
                m[8] = a2.x;
                jinvG = a2.y;
                csd2 = a2.z;
                rjG = a2.w;
                nrm[0] = a3.x;
                nrm[1] = a3.y;
                nrm[2] = a3.z;
            }
            const int gkL = gidx(kL, nk, pk);
            float qv[2][5];
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int f = 0; f < 5; ++f) qv[t][f] = 0.0f;
            if (SEP && !tmap) cp_async_wait_all();
            bool from_box = false;
            if (tmap && gkL >= 0) {
                // the box of this plane (issued one iteration earlier); a wait
                // that gives up is recorded (site 8) instead of hanging, and
                // this thread reads the plane from global memory
                if (mbar_wait(S.MBAR, tpar, wait_limit)) {
                    from_box = true;
                    tpar ^= 1u;
                } else {
                    if (J.oob) atomicCAS(J.oob, 0ull, 8ull << 48);
                    tma_off = true;
                    pend = true;
                }
            }
            if (gkL >= 0) {
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (lc[t] < 0) continue;
                    const long long o = CK_G(2, gkL * plane + lo2[t]);
                    if (from_box) {
#pragma unroll
                        for (int f = 0; f < 5; ++f)
                            qv[t][f] = S.QG[CK_TAB(f * (G_::C2Y * TMA_BOX_X) + qg[t], 5 * G_::C2Y * TMA_BOX_X)];
                    } else if (SEP && !tmap && !tma_off) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) qv[t][f] = S.QS[(t * 5 + f) * G_::NT + tid];
                    } else {
#pragma unroll
                        for (int f = 0; f < 5; ++f) qv[t][f] = Qs[f * fs + o];
                    }
                }
            }
            if (!SEP && g_act) {
                S.MA[CK_TAB((rG * 2 + 0) * N1 + c1, 4 * N1)] = make_float4(m[0], m[1], m[2], m[3]);
                S.MA[CK_TAB((rG * 2 + 1) * N1 + c1, 4 * N1)] = make_float4(m[4], m[5], m[6], m[7]);
                S.MB[CK_TAB(rG * N1 + c1, 2 * N1)] = make_float2(m[8], jinvG);
            }
            if (gkL >= 0) {
                const int sb = sl[5] * N2;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (lc[t] < 0) continue;
                    const float rho = qv[t][0];
                    const float rr = __fdividef(1.0f, rho);
                    const float u = qv[t][1] * rr, v = qv[t][2] * rr, w = qv[t][3] * rr;
                    const float e = qv[t][4];
                    const float p = FP.gm1 * (e - 0.5f * rho * (u * u + v * v + w * w));
                    S.PA[CK_RING(sb + lc[t])] = make_float4(rho, u, v, w);
                    S.PB[CK_RING(sb + lc[t])] = make_float2(p, FP.gam * p * rr);
                }
            }
            // (a thread whose staging wait gave up turns staging off for the
            // whole CTA here)
            tma_off = __syncthreads_or(tma_off) != 0;
            if (tma_off) tmap = nullptr;
            // the next plane's box, in flight during the rest of this iteration
            // (every thread has read this plane's box)
            if (tmap) stage_box(kL + 1);
            // ---- derivatives, SGS, sensors, lambda-bar of plane kG on R1 (one cell per thread) ----
            if (g_act) {
                const int s0 = CK_RING(sl[3] * N2 + c2); // plane kG
                const float4 A0 = S.PA[s0];
                const float2 B0 = S.PB[s0];
                D3 dd[3];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int st = a == 0 ? 1 : C2X;
                    const int tt = a == 0 ? ti : tj;
                    if (tt == 0) {
                        const int sm = CK_RING(s0 - st), sp = CK_RING(s0 + st);
                        dd[a] = deriv_central(S.PA[sm], S.PB[sm], B0.x, S.PA[sp], S.PB[sp]);
                    } else {
                        const int o1 = CK_RING(s0 + (tt - 1) * st), o2 = CK_RING(s0 + tt * st),
                                  o3 = CK_RING(s0 + (tt + 1) * st);
                        dd[a] = deriv_end(tt, S.PA[o1], S.PB[o1], S.PA[o2], S.PB[o2], S.PA[o3], S.PB[o3]);
                    }
                }
                {
                    // zeta stencil of this plane (uniform): central, or one-sided at an end
                    const int tk = (!pk && gkG == 0) ? 1 : ((!pk && gkG == nk - 1) ? -1 : 0);
                    if (tk == 0) {
                        const int om = CK_RING(sl[2] * N2 + c2), op = CK_RING(sl[4] * N2 + c2);
                        dd[2] = deriv_central(S.PA[om], S.PB[om], B0.x, S.PA[op], S.PB[op]);
                    } else {
                        const int o1 = CK_RING(sl[tk > 0 ? 3 : 1] * N2 + c2), o2 = CK_RING(sl[tk > 0 ? 4 : 2] * N2 + c2),
                                  o3 = CK_RING(sl[tk > 0 ? 5 : 3] * N2 + c2);
                        dd[2] = deriv_end(tk, S.PA[o1], S.PB[o1], S.PA[o2], S.PB[o2], S.PA[o3], S.PB[o3]);
                    }
                }
                // physical velocity gradient by the chain rule, |S|, Smagorinsky mu_sgs
                float gu[3][3];
                float rh[3];
                if constexpr (SEP) {
                    const float4 hX = S.HX[tx + 1], hY = S.HY[ty + 1], hZ = F.h1[2][gkG];
                    rh[0] = hX.y;
                    rh[1] = hY.y;
                    rh[2] = hZ.y;
                    csd2 = FP.cs2 * hX.z * hY.z * hZ.z;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) gu[i][cc] = cmp(dd[cc].d, i) * rh[cc];
                } else {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc)
                            gu[i][cc] = (m[cc] * cmp(dd[0].d, i) + m[3 + cc] * cmp(dd[1].d, i) +
                                         m[6 + cc] * cmp(dd[2].d, i)) * rjG;
                }
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
                const float rho = A0.x, T = B0.y;
                const float mus = rho * csd2 * sqrt_nonneg(2.0f * ss);
                const float sT = sqrt_pos(T);
                const float mu = __fdividef(T * sT * FP.suth1, T + FP.suthS);
                float lam[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if constexpr (SEP) {
                        lam[a] = (fabsf(cmp(A0, 1 + a)) + sT) * fabsf(rh[a]);
                    } else {
                        const float JU = m[3 * a] * A0.y + m[3 * a + 1] * A0.z + m[3 * a + 2] * A0.w;
                        lam[a] = (fabsf(JU) + sT * nrm[a]) * rjG;
                    }
                }
                const float s01 = sqrt_nonneg(lam[0] * lam[1]), s02 = sqrt_nonneg(lam[0] * lam[2]),
                            s12 = sqrt_nonneg(lam[1] * lam[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a) S.GD[CK_TAB((rG * 3 + a) * N1 + c1, 6 * N1)] = dd[a].d;
                S.GC[CK_TAB((rG * 2 + 0) * N1 + c1, 4 * N1)] = make_float4(mu * FP.inv_Re + mus, mu * FP.kap_mol + mus * FP.kap_sgs,
                                                           dd[0].nu, lam[0] + s01 + s02);
                S.GC[CK_TAB((rG * 2 + 1) * N1 + c1, 4 * N1)] = make_float4(dd[1].nu, lam[1] + s01 + s12, dd[2].nu, lam[2] + s02 + s12);
            }
            // No barrier here: the interfaces below read the R1 tables of plane
            // kG only in this thread's own column (the zeta neighbour), written
            // just above by this thread; everything they read from other
            // threads (plane kU tables, the point ring) was written before the
            // previous iteration's closing barrier, and the phase writes only
            // plane-kG slots, which no interface of this iteration reads.
            if (SEP && !tmap && !tma_off) {
                // next plane's state, in flight during the interface arithmetic
                stage_q(kL + 1);
                cp_async_commit();
            }
            // ---- interfaces and update of plane kU = kL - 3 ----
            const int kU = kL - 3;
            if (kU >= k0 - 1) {
                const int gk = gidx(kU, nk, pk);
                const bool plane_ok = gk >= 0;
                const bool first = kU == k0 - 1; // only the -1/2 zeta flux of the chunk
                const bool do_xi = !first && plane_ok && xi_ok;
                const bool do_eta = !first && plane_ok && eta_ok;
                const bool do_zeta = plane_ok && out_col && (pk || gk < nk - 1);
                const bool upd = !first && plane_ok && out_col && kU < k1;
                const long long o = CK_G(4, (long long)(plane_ok ? gk : 0) * plane + ocol);
                // separable form: Q(0) of the updated point, in flight during the interfaces
                float q0s[5] = {0, 0, 0, 0, 0};
                if (SEP && upd && !rhs_only) {
                    const float *Q0 = J.q[0];
#pragma unroll
                    for (int f = 0; f < 5; ++f) q0s[f] = Q0[f * fs + o];
                }
                const int rU = ring2(kU), sU = sl[2] * N2;
                OwnPt L;
                if (do_xi || do_eta || do_zeta) {
                    L.a = S.PA[sU + c2];
                    {
                        const float2 b = S.PB[sU + c2];
                        L.p = b.x;
                        L.T = b.y;
                    }
                    if constexpr (!SEP) {
                        const float4 u0 = S.MA[CK_TAB((rU * 2 + 0) * N1 + c1, 4 * N1)],
                                     u1 = S.MA[CK_TAB((rU * 2 + 1) * N1 + c1, 4 * N1)];
                        const float2 u2 = S.MB[CK_TAB(rU * N1 + c1, 2 * N1)];
                        L.m[0] = u0.x; L.m[1] = u0.y; L.m[2] = u0.z; L.m[3] = u0.w;
                        L.m[4] = u1.x; L.m[5] = u1.y; L.m[6] = u1.z; L.m[7] = u1.w;
                        L.m[8] = u2.x;
                        L.jinv = u2.y;
                    }
                    L.c1 = c1;
                    L.pl = rU;
                }
                // residual R = sum over axes of (flux(+1/2) - flux(-1/2)); the
                // -1/2 xi flux comes from the lane below, the -1/2 zeta flux
                // from the previous plane, the -1/2 eta flux (row below)
                // through shared memory after the barrier
                float R[5], hy[5] = {0, 0, 0, 0, 0};
                {
                    float hx[5] = {0, 0, 0, 0, 0};
                    if (do_xi) {
                        if constexpr (SEP) {
                            const float4 hX = S.HX[tx + 1], hY = S.HY[ty + 1], hZ = F.h1[2][gk];
                            fused_iface_sep<0, TY>(S, FP, L, CK_RING(sU + c2 + 1), CK_RING(sU + c2 - 1),
                                                   CK_RING(sU + c2 + 2), CK_TAB(c1 + 1, N1), rU,
                                                   xi_lo, xi_hi, hX.x, S.HX[tx + 2].x, hY.x, hY.y, hZ.x, hZ.y, hx);
                        } else {
                            fused_iface<0, TY>(S, FP, L, CK_RING(sU + c2 + 1), CK_RING(sU + c2 - 1),
                                               CK_RING(sU + c2 + 2), CK_TAB(c1 + 1, N1), rU, xi_lo,
                                               xi_hi, hx);
                        }
                    }
#pragma unroll
                    for (int f = 0; f < 5; ++f) R[f] = hx[f] - __shfl_up_sync(0xffffffffu, hx[f], 1);
                }
                if (do_eta) {
                    if constexpr (SEP) {
                        const float4 hX = S.HX[tx + 1], hY = S.HY[ty + 1], hZ = F.h1[2][gk];
                        fused_iface_sep<1, TY>(S, FP, L, CK_RING(sU + c2 + C2X), CK_RING(sU + c2 - C2X),
                                               CK_RING(sU + c2 + 2 * C2X), CK_TAB(c1 + FX, N1),
                                               rU, eta_lo, eta_hi, hY.x, S.HY[ty + 2].x, hX.x, hX.y, hZ.x, hZ.y, hy);
                    } else {
                        fused_iface<1, TY>(S, FP, L, CK_RING(sU + c2 + C2X), CK_RING(sU + c2 - C2X),
                                           CK_RING(sU + c2 + 2 * C2X), CK_TAB(c1 + FX, N1), rU,
                                           eta_lo, eta_hi, hy);
                    }
                }
#pragma unroll
                for (int f = 0; f < 5; ++f) S.SH[CK_SH((f * TY + ty) * FX + tx)] = hy[f];
                {
                    float hz[5] = {0, 0, 0, 0, 0};
                    if (do_zeta) {
                        const bool lo = !pk && gk == 0, hi = !pk && gk + 1 == nk - 1;
                        if constexpr (SEP) {
                            const float4 hX = S.HX[tx + 1], hY = S.HY[ty + 1], hZ = F.h1[2][gk];
                            const float hZR = F.h1[2][gidx(kU + 1, nk, pk)].x;
                            fused_iface_sep<2, TY>(S, FP, L, CK_RING(sl[3] * N2 + c2), CK_RING(sl[1] * N2 + c2),
                                                   CK_RING(sl[4] * N2 + c2), c1,
                                                   ring2(kU + 1), lo, hi, hZ.x, hZR, hX.x, hX.y, hY.x, hY.y, hz);
                        } else {
                            fused_iface<2, TY>(S, FP, L, CK_RING(sl[3] * N2 + c2), CK_RING(sl[1] * N2 + c2),
                                               CK_RING(sl[4] * N2 + c2), c1,
                                               ring2(kU + 1), lo, hi, hz);
                        }
                    }
#pragma unroll
                    for (int f = 0; f < 5; ++f) {
                        R[f] += hz[f] - hz_prev[f];
                        hz_prev[f] = hz[f];
                    }
                }
                // Q(0) of the updated point, requested before the exchange barrier
                float q0v[5] = {0, 0, 0, 0, 0};
                if (!SEP && upd && !rhs_only) {
                    const float *Q0 = J.q[0];
#pragma unroll
                    for (int f = 0; f < 5; ++f) q0v[f] = Q0[f * fs + o];
                }
                __syncthreads();
                if (upd) {
#pragma unroll
                    for (int f = 0; f < 5; ++f) R[f] += hy[f] - S.SH[CK_SH((f * TY + ty - 1) * FX + tx)];
                    if (rhs_only) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) J.rhs[f * fs + o] = R[f];
                    } else {
                        if constexpr (SEP) {
#pragma unroll
                            for (int f = 0; f < 5; ++f) q0v[f] = q0s[f];
                        }
                        float rjk;
                        if constexpr (SEP) {
                            rjk = S.HX[tx + 1].y * S.HY[ty + 1].y * F.h1[2][gk].y;
                        } else {
                            rjk = rjU;
                        }
                        const float adtj = adt * rjk;
#pragma unroll
                        for (int f = 0; f < 5; ++f) Qd[f * fs + o] = q0v[f] - adtj * R[f];
                    }
                }
            }
            if constexpr (!SEP) rjU = rjG; // plane kG is the next iteration's kU
            __syncthreads();
        }
    }
    // a copy whose wait gave up may still be in flight into this CTA's
    // shared memory: its issuer waits for it (bounded) before exiting; if
    // that wait gives up too, the copy may land in the shared memory of the
    // next CTA on this SM, which is recorded as site 9 (it outranks site 8:
    // the state can no longer be trusted)
    if (pend && tid == 0 && !mbar_wait(S.MBAR, tpar, MBAR_WAIT_LIMIT)) {
        const JetDev<float> &J0 = jets[0];
        if (J0.oob) atomicMax(J0.oob, 9ull << 48);
    }
}

#undef CK_G
#undef CK_RING
#undef CK_TAB
#undef CK_SH

template <int TY> int fused_prepare()
{
    int rc = (int)cudaFuncSetAttribute(k_fused<TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Geo<TY>::BYTES_GEN);
    if (rc) return rc;
    return (int)cudaFuncSetAttribute(k_fused<TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Geo<TY>::BYTES_SEP);
}

template <int TY>
void launch_fused(const JetDev<float> *jets, const FusedJet *fj, int njets, int total_items, int total_tiles,
                  int grid, int src, int dst, int stage, const double *dt, int rhs_only, int separable, int balanced,
                  int wait_limit, cudaStream_t st)
{
    dim3 block(FX, TY);
    if (wait_limit < 0) wait_limit = MBAR_WAIT_LIMIT;
    if (separable)
        k_fused<TY, true><<<grid, block, Geo<TY>::BYTES_SEP, st>>>(jets, fj, njets, total_items, total_tiles, src,
                                                              dst, stage, dt, rhs_only, balanced, wait_limit);
    else
        k_fused<TY, false><<<grid, block, Geo<TY>::BYTES_GEN, st>>>(jets, fj, njets, total_items, total_tiles, src,
                                                               dst, stage, dt, rhs_only, balanced, wait_limit);
}

template int fused_prepare<16>();
template int fused_prepare<8>();
template void launch_fused<16>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int, int,
                               const double *, int, int, int, int, cudaStream_t);
template void launch_fused<8>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int, int,
                              const double *, int, int, int, int, cudaStream_t);

} // namespace les
