// Fused single-pass Runge-Kutta stage for FP32 storage and arithmetic.
//
// One kernel does what k_point, k_grads, k_iface and k_update do for the FP64
// path (Secs. "Numerical Formulation", "Time Marching Method"), with the
// intermediate per-point and per-interface quantities in shared memory and
// registers instead of HBM: per stage a point's state, Q(0) and static metrics
// are read and its new state written once.
//
// Row pairs and paired arithmetic.  A CTA of 32 x TY/2 threads owns a tile of
// 32 columns x TY rows (region R1) and updates its 30 x (TY-2) inner points.
// Thread (tx, tr) owns the two points of column tx in rows 2tr and 2tr+1 and
// evaluates everything of the two points together: each quantity is a float2
// whose lanes are the two rows, and the arithmetic runs as paired FP32
// instructions (add/mul/fma .f32x2, two results per issue).  Shared-memory
// records interleave the two rows the same way, so one 16-byte load yields two
// quantities of both points in register pairs.  The interfaces to the +xi and
// +zeta neighbours pair up row by row; the two +eta interfaces of a thread
// (rows 2tr|2tr+1 and 2tr+1|2tr+2) take their right-hand points from its own
// second row and the next thread row's first.
//
// Halo.  Point data (primitives and rho H) live in a ring of 4 planes over
// R2 = R1 plus one column on each side and two rows above and below; cells
// outside a non-periodic axis hold the mirror image of the point one beyond
// the boundary point (W(-1) = W(1), W(n) = W(n-2)), which is the paper's
// boundary fourth difference, so the interface arithmetic has no end cases.
// Derivatives, transport coefficients, sensors, lambda-bar and metric
// cofactors of R1 are kept for two planes.  Per loaded plane kL:
// primitives(kL) | gradients(kL-1) | interfaces + update(kL-2).  The
// gradients of the first plane of a non-periodic k axis, which need planes
// 0..2, are formed one plane late, together with plane 1.
//
// Work list.  Items (jet, tile x, tile y, k-chunk) are walked by a persistent
// grid in a fixed order; results do not depend on the item order, the chunk
// length or the grid size: every point is computed by the same instruction
// sequence whichever tile, lane or chunk it falls in.
#include <algorithm>
#include <cmath>

#include "les_internal.cuh"

namespace les {

namespace {

constexpr int FX = 32; // threads (grid columns) along i

__constant__ float c_alpha_f[5] = {0.25f, 1.0f / 6.0f, 0.375f, 0.5f, 1.0f};

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic (two rows per register pair)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once like a scalar subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc(-1.0f), a); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// the pair (second lane of a, first lane of b): the +eta neighbours of a
// thread's two rows
__device__ __forceinline__ float2 odd2(float2 a, float2 b) { return make_float2(a.y, b.x); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
// hardware approximate reciprocal (positive, normal arguments)
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y)); }
// square root of x >= 0 through the hardware reciprocal square root
// (max. 2 ulp): x * rsqrt(x), 0 -> 0 (a spectral radius vanishes on the axis
// of a polar mesh)
__device__ __forceinline__ float2 sqrt2(float2 x)
{
    return mul2(x, make_float2(rsqrtf(fmaxf(x.x, 1.17549435e-38f)), rsqrtf(fmaxf(x.y, 1.17549435e-38f))));
}

// ---------------------------------------------------------------------------
// Shared-memory map (byte offsets; 16-byte records first)
//   ring (3 planes; 4 separable) over R2 pair cells:  PA (rho, u)  PB (v, w)  PC (p, T)
//                                         float4 each; PH (rho H) float2
//   R1 tables (2 planes) over R1 pair cells:
//     GD [3 axes][2]  float4: 2 d/d xi^a of (u, v) and (w, T)
//     GC [4]          float4: (mu_eff, kappa), (nu_a, lambda-bar_a) a = 0..2
//   MA [3 planes][5] float4 over R1 pair cells: cofactors (m0 m1) (m2 m3)
//                             (m4 m5) (m6 m7) (m8 J^-1), streamed in by
//                             cp.async one plane ahead (general form only)
//   SH [5][NT] float          eta flux of each thread's second row
//   QZ [5][TY-2][30] float    Q(0) of the tile's updated points, copied in
//                             by cp.async during the plane's iteration
//   HX [C2], HY [TY+4] float4 separable form: (h, 1/h, h^(2/3), 0) of the
//                             tile's columns / rows
//   HZ [4] float4             separable form: the same for planes k (slot k & 3),
//                             copied in two planes ahead
//   QG [5][TY+4][40] float    the next plane's state box (TMA), 128-aligned,
//                             then its mbarrier
// A "pair cell" is one column of two rows (2p, 2p+1); its float4 records
// interleave the two rows: (q1(2p), q1(2p+1), q2(2p), q2(2p+1)).
// ---------------------------------------------------------------------------
template <int TY, bool SEP> struct Geo {
    static constexpr int TR = TY / 2;              // thread rows
    static constexpr int NT = FX * TR;             // threads
    static constexpr int C2 = FX + 2;              // R2 columns -1 .. FX
    static constexpr int P2 = TR + 2;              // R2 pair rows -1 .. TR (rows -2 .. TY+1)
    static constexpr int N2 = C2 * P2;             // R2 pair cells
    static constexpr int N1 = NT;                  // R1 pair cells
    static constexpr int BR = tma_box_rows(TY);    // rows of the staging box
    // planes of the point ring: 3 in the general form (its shared memory
    // also holds three planes of metric records), 4 in the separable form
    static constexpr int NR = SEP ? 4 : 3;
    static constexpr size_t O_PA = 0;
    static constexpr size_t O_PB = O_PA + 16ull * NR * N2;
    static constexpr size_t O_PC = O_PB + 16ull * NR * N2;
    static constexpr size_t O_PH = O_PC + 16ull * NR * N2;
    static constexpr size_t O_GD = O_PH + 8ull * NR * N2;
    static constexpr size_t O_GC = O_GD + 16ull * 2 * 6 * N1;
    static constexpr size_t O_MA = O_GC + 16ull * 2 * 4 * N1;
    static constexpr size_t O_SH = O_MA + (SEP ? 0ull : 16ull * 3 * 5 * N1);
    static constexpr int QZN = (TY - 2) * (FX - 2); // updated points of a tile plane
    static constexpr size_t O_QZ = (O_SH + 4ull * 5 * NT + 15) / 16 * 16;
    static constexpr size_t O_HX = O_QZ + 4ull * 5 * QZN;
    // (the spacing tables exist in the separable form only)
    static constexpr size_t O_HY = O_HX + (SEP ? 16ull * C2 : 0ull);
    static constexpr size_t O_HZ = O_HY + (SEP ? 16ull * BR : 0ull);
    static constexpr size_t O_QG = (O_HZ + (SEP ? 16ull * 4 : 0ull) + 127) / 128 * 128;
    static constexpr unsigned BOX_BYTES = 4u * 5 * BR * TMA_BOX_X;
    static_assert(BOX_BYTES % 16 == 0, "box size");
    static constexpr size_t O_MBAR = O_QG + BOX_BYTES;
    static constexpr size_t O_FPS = O_MBAR + 8;
    static constexpr size_t BYTES = O_FPS + 64;
    static_assert(BYTES <= 227 * 1024, "shared memory of one CTA");
};

template <int TY, bool SEP> struct Sm {
    float4 *PA, *PB, *PC;
    float2 *PH;
    float4 *GD, *GC, *MA;
    float *SH, *QZ;
    float4 *HX, *HY, *HZ;
    float *QG;
    unsigned long long *MBAR;
    float *FPS; // a batch jet's constants (FusedParams) for the item
    __device__ __forceinline__ explicit Sm(unsigned char *b)
        : PA((float4 *)(b + Geo<TY, SEP>::O_PA)), PB((float4 *)(b + Geo<TY, SEP>::O_PB)),
          PC((float4 *)(b + Geo<TY, SEP>::O_PC)), PH((float2 *)(b + Geo<TY, SEP>::O_PH)),
          GD((float4 *)(b + Geo<TY, SEP>::O_GD)), GC((float4 *)(b + Geo<TY, SEP>::O_GC)),
          MA((float4 *)(b + Geo<TY, SEP>::O_MA)), SH((float *)(b + Geo<TY, SEP>::O_SH)),
          QZ((float *)(b + Geo<TY, SEP>::O_QZ)),
          HX((float4 *)(b + Geo<TY, SEP>::O_HX)), HY((float4 *)(b + Geo<TY, SEP>::O_HY)),
          HZ((float4 *)(b + Geo<TY, SEP>::O_HZ)),
          QG((float *)(b + Geo<TY, SEP>::O_QG)), MBAR((unsigned long long *)(b + Geo<TY, SEP>::O_MBAR)),
          FPS((float *)(b + Geo<TY, SEP>::O_FPS))
    {
    }
};

// Slot of plane k (k >= -6) in the three-plane rings.
__device__ __forceinline__ int r3(int k) { return (k + 6) % 3; }
// Slot of plane k in the point ring of NR planes.
template <int NR> __device__ __forceinline__ int rslot(int k) { return NR == 4 ? (k & 3) : r3(k); }

// Asynchronous 16-byte global -> shared copy, not kept in L1 (completes
// without the issuing thread waiting; cp_async_wait_prev() waits for all of
// this thread's groups but the most recent one).
__device__ __forceinline__ unsigned smem_u32_(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32_(dst)), "l"(src) : "memory");
}
// 4-byte variant (scattered Q(0) values)
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32_(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Index of a tile cell along an axis: wrapped on a periodic axis; on a
// non-periodic one the mirror image about the end point (-g, 2(n-1) - g),
// clamped into the axis for cells further out (those feed no result).
__device__ __forceinline__ int map_idx(int g, int n, int per)
{
    if (per) {
        const int h = g < 0 ? g + n : (g >= n ? g - n : g);
        return (unsigned)h < (unsigned)n ? h : wrapi(g, n);
    }
    const int m = g < 0 ? -g : (g > n - 1 ? 2 * (n - 1) - g : g);
    return m < 0 ? 0 : (m > n - 1 ? n - 1 : m);
}

// TMA staging: an mbarrier with one arrival (the issuing thread's, carrying
// the expected byte count) completed by the copy.
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

// Point data of one side of an interface: two points (the two lanes).
struct Pts {
    float2 rho, u, v, w, p, T, rH; // rH = rho H = e + p
};
__device__ __forceinline__ Pts odd_pts(const Pts &a, const Pts &b)
{
    Pts r;
    r.rho = odd2(a.rho, b.rho);
    r.u = odd2(a.u, b.u);
    r.v = odd2(a.v, b.v);
    r.w = odd2(a.w, b.w);
    r.p = odd2(a.p, b.p);
    r.T = odd2(a.T, b.T);
    r.rH = odd2(a.rH, b.rH);
    return r;
}
// Dissipation vector W = [rho, rho u, rho v, rho w, e + p] (Eq. W_dissip,
// with the unscaled conserved variables)
__device__ __forceinline__ void wvec(const Pts &q, float2 W[5])
{
    W[0] = q.rho;
    W[1] = mul2(q.rho, q.u);
    W[2] = mul2(q.rho, q.v);
    W[3] = mul2(q.rho, q.w);
    W[4] = q.rH;
}

// Transport data of one side: coefficients, sensor and lambda-bar along the
// interface axis, and the doubled derivatives 2 d/d xi^b of (u, v, w, T)
// along the two tangential axes b (ascending).
struct Side {
    float2 mue, kap, nu, lb;
    float2 d[2][4];
};

// Flux through the interfaces between the points L and their +A neighbours R
// (Eqs. spatial_discret, inv_flux_vec, dissip_term, eps_2/4_dissip; the
// compact viscous + SGS flux of the interface): the centred inviscid flux
// minus J^-1 d minus the viscous flux, general metric cofactors.  WLm, WRp:
// W of the outer points of the dissipation stencil.
template <int A>
__device__ __forceinline__ void iface(const FusedParams &FP, const Pts &L, const float2 WL[5], const float2 mL[9],
                                      float2 jL, const Pts &R, const float2 WR[5], const float2 mR[9], float2 jR,
                                      const float2 WLm[5], const float2 WRp[5], const Side &SL, const Side &SR,
                                      float2 H[5])
{
    const float2 half = bc(0.5f);
    // centred inviscid flux: J^-1 U = m_A . u; the ambient pressure is taken
    // out of the pressure terms (a constant pressure has no flux divergence,
    // and leaving it in adds FP32 rounding of O(1) terms to small momentum
    // residuals)
    const float2 hJL = mul2(half, fma2(mL[3 * A + 2], L.w, fma2(mL[3 * A + 1], L.v, mul2(mL[3 * A], L.u))));
    const float2 hJR = mul2(half, fma2(mR[3 * A + 2], R.w, fma2(mR[3 * A + 1], R.v, mul2(mR[3 * A], R.u))));
    const float2 hpinf = bc(-0.5f * FP.pinf);
    const float2 pl = fma2(L.p, half, hpinf), pr = fma2(R.p, half, hpinf);
    H[0] = fma2(WR[0], hJR, mul2(WL[0], hJL));
#pragma unroll
    for (int c = 0; c < 3; ++c)
        H[1 + c] = fma2(pr, mR[3 * A + c], fma2(pl, mL[3 * A + c], fma2(WR[1 + c], hJR, mul2(WL[1 + c], hJL))));
    H[4] = fma2(WR[4], hJR, mul2(WL[4], hJL));
    // Turkel-Vatsa dissipation: F += se4 (W(R+1) - W(L-1)) - (se2 + 3 se4)(W(R) - W(L))
    const float2 Js = add2(jL, jR); // 2 x interface J^-1
    {
        const float2 eps2 = mul2(bc(FP.k2), max2(SL.nu, SR.nu));
        const float2 eps4 = max2(bc(0.0f), sub2(bc(FP.k4), eps2));
        const float2 sc = mul2(mul2(bc(0.25f), Js), add2(SL.lb, SR.lb));
        const float2 se4 = mul2(sc, eps4);
        const float2 c2 = fma2(se4, bc(3.0f), mul2(sc, eps2));
#pragma unroll
        for (int f = 0; f < 5; ++f) H[f] = fma2(c2, sub2(WL[f], WR[f]), fma2(se4, sub2(WRp[f], WLm[f]), H[f]));
    }
    // compact viscous + SGS flux.  With Ms = m_L + m_R (twice the interface
    // cofactors) and D = 4 x the computational derivatives at the interface
    // (normal: 4 (phi_R - phi_L); tangential: the sum of the two points'
    // doubled central differences), G_fc = sum_b Ms_bc D_fb = 4 Js d phi_f / d x_c.
    // Only row A of the stress tensor is needed:
    //   s_i = coef/(16 Js) (X_i + Y_i - 2/3 Ms_Ai div),  coef = mu_eff,L + mu_eff,R
    //   X_f = sum_c Ms_Ac G_fc = sum_b K_b D_fb,  K_b = sum_c Ms_Ac Ms_bc
    //   Y_i = sum_c Ms_Ac G_ci = sum_b Ms_bi w_b,  w_b = sum_c Ms_Ac D_cb
    //   div = sum_i G_ii
    // and the energy flux is s . u_interface + (kappa_L + kappa_R) X_T / (16 Js).
    {
        constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
        float2 Ms[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) Ms[t] = add2(mL[t], mR[t]);
        float2 D[4][3];
        const float2 four = bc(4.0f);
        D[0][A] = mul2(four, sub2(R.u, L.u));
        D[1][A] = mul2(four, sub2(R.v, L.v));
        D[2][A] = mul2(four, sub2(R.w, L.w));
        D[3][A] = mul2(four, sub2(R.T, L.T));
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            D[f][B1] = add2(SL.d[0][f], SR.d[0][f]);
            D[f][B2] = add2(SL.d[1][f], SR.d[1][f]);
        }
        float2 K[3], wv[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            K[b] = fma2(Ms[3 * A + 2], Ms[3 * b + 2], fma2(Ms[3 * A + 1], Ms[3 * b + 1], mul2(Ms[3 * A], Ms[3 * b])));
            wv[b] = fma2(Ms[3 * A + 2], D[2][b], fma2(Ms[3 * A + 1], D[1][b], mul2(Ms[3 * A], D[0][b])));
        }
        float2 X[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) X[f] = fma2(K[2], D[f][2], fma2(K[1], D[f][1], mul2(K[0], D[f][0])));
        float2 dv = mul2(Ms[0], D[0][0]);
        dv = fma2(Ms[3], D[0][1], dv);
        dv = fma2(Ms[6], D[0][2], dv);
        dv = fma2(Ms[1], D[1][0], dv);
        dv = fma2(Ms[4], D[1][1], dv);
        dv = fma2(Ms[7], D[1][2], dv);
        dv = fma2(Ms[2], D[2][0], dv);
        dv = fma2(Ms[5], D[2][1], dv);
        dv = fma2(Ms[8], D[2][2], dv);
        const float2 rJ = rcp2(Js);
        const float2 f1 = mul2(mul2(add2(SL.mue, SR.mue), rJ), bc(1.0f / 16.0f));
        const float2 ntd = mul2(mul2(f1, bc(-2.0f / 3.0f)), dv);
        float2 s[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float2 Y = fma2(Ms[6 + i], wv[2], fma2(Ms[3 + i], wv[1], mul2(Ms[i], wv[0])));
            s[i] = fma2(Ms[3 * A + i], ntd, mul2(f1, add2(X[i], Y)));
            H[1 + i] = sub2(H[1 + i], s[i]);
        }
        const float2 kh = mul2(mul2(add2(SL.kap, SR.kap), rJ), bc(1.0f / 16.0f));
        const float2 e = fma2(s[2], add2(L.w, R.w), fma2(s[1], add2(L.v, R.v), mul2(s[0], add2(L.u, R.u))));
        H[4] = sub2(H[4], fma2(kh, X[3], mul2(half, e)));
    }
}

// Separable form of iface on a Cartesian-product grid x = x(i), y = y(j),
// z = z(k) (Sec. "Transformation of Coordinates" with diagonal metrics): the
// cofactor matrix is diag(y_eta z_zeta, x_xi z_zeta, x_xi y_eta), so the face
// factor Sa of axis A is the product of the two tangential spacings (equal on
// both sides), the interface J^-1 is Sa hb with hb the average spacing along
// A, and the chain rule is d/dx_c = (1/h_c) d/dxi_c.  rhb = 1/hb; rq1, rq2:
// 1/4 of the reciprocal tangential spacings (axes B1 < B2), which turn the
// sums of doubled differences into derivatives.
template <int A>
__device__ __forceinline__ void iface_sep(const FusedParams &FP, const Pts &L, const float2 WL[5], const Pts &R,
                                          const float2 WR[5], const float2 WLm[5], const float2 WRp[5],
                                          const Side &SL, const Side &SR, float2 Sa, float2 hb, float2 rhb,
                                          float2 rq1, float2 rq2, float2 H[5])
{
    const float2 half = bc(0.5f);
    const float2 hS = mul2(half, Sa);
    // centred inviscid flux: J^-1 U_A = Sa u_A on both sides
    const float2 uAL = A == 0 ? L.u : (A == 1 ? L.v : L.w), uAR = A == 0 ? R.u : (A == 1 ? R.v : R.w);
    const float2 hJL = mul2(hS, uAL), hJR = mul2(hS, uAR);
#pragma unroll
    for (int f = 0; f < 5; ++f) H[f] = fma2(WR[f], hJR, mul2(WL[f], hJL));
    H[1 + A] = fma2(hS, sub2(add2(L.p, R.p), bc(2.0f * FP.pinf)), H[1 + A]); // ambient pressure out, as above
    // Turkel-Vatsa dissipation
    {
        const float2 eps2 = mul2(bc(FP.k2), max2(SL.nu, SR.nu));
        const float2 eps4 = max2(bc(0.0f), sub2(bc(FP.k4), eps2));
        const float2 sc = mul2(mul2(hS, hb), add2(SL.lb, SR.lb)); // Sa hb (lb_L + lb_R) / 2
        const float2 se4 = mul2(sc, eps4);
        const float2 c2 = fma2(se4, bc(3.0f), mul2(sc, eps2));
#pragma unroll
        for (int f = 0; f < 5; ++f) H[f] = fma2(c2, sub2(WL[f], WR[f]), fma2(se4, sub2(WRp[f], WLm[f]), H[f]));
    }
    // compact viscous + SGS flux: only row A of the stress tensor is needed
    {
        float2 g[4][3]; // physical gradient of (u, v, w, T) at the interface
        constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
        g[0][A] = mul2(sub2(R.u, L.u), rhb);
        g[1][A] = mul2(sub2(R.v, L.v), rhb);
        g[2][A] = mul2(sub2(R.w, L.w), rhb);
        g[3][A] = mul2(sub2(R.T, L.T), rhb);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            g[f][B1] = mul2(add2(SL.d[0][f], SR.d[0][f]), rq1);
            g[f][B2] = mul2(add2(SL.d[1][f], SR.d[1][f]), rq2);
        }
        const float2 coef = mul2(half, add2(SL.mue, SR.mue)); // mu_eff at the interface
        const float2 dv3 = mul2(bc(2.0f / 3.0f), add2(add2(g[0][0], g[1][1]), g[2][2]));
        float2 tA[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
            tA[i] = i == A ? mul2(coef, sub2(add2(g[A][A], g[A][A]), dv3)) : mul2(coef, add2(g[A][i], g[i][A]));
        const float2 kap = mul2(half, add2(SL.kap, SR.kap));
#pragma unroll
        for (int i = 0; i < 3; ++i) H[1 + i] = sub2(H[1 + i], mul2(Sa, tA[i]));
        const float2 e = fma2(tA[2], add2(L.w, R.w), fma2(tA[1], add2(L.v, R.v), mul2(tA[0], add2(L.u, R.u))));
        H[4] = sub2(H[4], mul2(Sa, fma2(kap, g[3][A], mul2(half, e))));
    }
}

} // namespace

// Index checks of a LES_BOUNDS_CHECK build (nothing otherwise): global
// offsets against their arrays (site 2 state, 3 static records, 4 update),
// shared-memory slots against their tables (5 point ring, 6 R1 tables and
// the staging box, 7 eta-flux rows).
#define CK_G(site, x, n) LES_BOUNDS(J.oob, (site), (x), (n))
#define CK_RING(x) ((int)LES_BOUNDS(J.oob, 5, (x), NRING * N2))
#define CK_TAB(x, n) ((int)LES_BOUNDS(J.oob, 6, (x), (n)))
#define CK_SH(x) ((int)LES_BOUNDS(J.oob, 7, (x), 5 * NT))

// The jet's table entries: in the single-jet form (ONE) the kernel
// parameters, whose fields the compiler reads from the parameter bank
// (warp-uniform operands, no memory loads in the plane loop); else the
// device tables.
template <bool ONE, typename T> __device__ __forceinline__ const T &jet_entry(const T &one, const T *tab, int j)
{
    if constexpr (ONE) return one;
    else return tab[j];
}

// The jet's constants: the kernel parameter (ONE), else the item's copy in
// shared memory (read with broadcast loads instead of global loads).
template <bool ONE>
__device__ __forceinline__ const FusedParams &jet_params(const FusedParams &param, const float *staged)
{
    if constexpr (ONE) return param;
    else return *reinterpret_cast<const FusedParams *>(staged);
}
static_assert(sizeof(FusedParams) % 4 == 0 && sizeof(FusedParams) <= 64, "FusedParams staging");

template <int TY, bool SEP, bool ONE>
__global__ void __launch_bounds__(FX * TY / 2, 1)
    k_fused(const JetDev<float> *__restrict__ jets, const FusedJet *__restrict__ fj, int njets,
            int total_items, int total_tiles, int src, int dst, int stage, const double *__restrict__ dt,
            int rhs_only, int balanced, int wait_limit, const __grid_constant__ JetDev<float> j1,
            const __grid_constant__ FusedJet f1)
{
    using G_ = Geo<TY, SEP>;
    constexpr int TR = G_::TR, NT = G_::NT, C2 = G_::C2, N2 = G_::N2, N1 = G_::N1, BR = G_::BR;
    constexpr int NRING = G_::NR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Sm<TY, SEP> S(smem_raw);
    const int tx = threadIdx.x, tr = threadIdx.y;
    const int tid = tr * FX + tx;
    const int c1 = tid;                       // own R1 pair cell
    const int c2 = (tr + 1) * C2 + (tx + 1);  // own R2 pair cell

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
    int item = blockIdx.x, w = 0, wend = 0;
    const int nwave = balanced == 2 ? total_tiles / (int)gridDim.x : 0;
    int wave = 0;
    auto jet_of_tile = [&](int t) {
        if constexpr (ONE) return 0;
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
                const FusedJet &Fw = jet_entry<ONE>(f1, fj, jet_of_tile(t));
                w = Fw.item0 + (t - Fw.tile0) * Fw.nkc;
                wend = w + Fw.nkc;
            } else {
                const int t1 = nwave * gridDim.x;
                int i1 = total_items;
                if (t1 < total_tiles) {
                    const FusedJet &Fw = jet_entry<ONE>(f1, fj, jet_of_tile(t1));
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
        if constexpr (!ONE) {
            int lo = 0, hi = njets;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (fj[mid].item0 <= key) lo = mid; else hi = mid;
            }
            jet = lo;
        }
        const JetDev<float> &J = jet_entry<ONE>(j1, jets, jet);
        const FusedJet &F = jet_entry<ONE>(f1, fj, jet);
        if constexpr (!ONE) {
            // staged for the item (the previous item's last reads of FPS
            // precede its closing barrier; the item barrier below publishes it)
            constexpr int NFP = sizeof(FusedParams) / 4;
            if (tid >= NT - NFP) S.FPS[tid - (NT - NFP)] = reinterpret_cast<const float *>(&F.fp)[tid - (NT - NFP)];
        }
        const FusedParams &FP = jet_params<ONE>(F.fp, S.FPS);
        const int ni = J.n[0], nj = J.n[1], nk = J.n[2];
        const int pi = J.per[0], pj = J.per[1], pk = J.per[2];
        // output ranges; on a periodic j axis the tiles start at row 1 (so that
        // their row pairs start on even rows) and the last one wraps to row 0
        const int ilo = pi ? 0 : 1, ihi = pi ? ni : ni - 1;
        const int jlo = 1, jhi = pj ? nj + 1 : nj - 1;
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
        const int ib = i0 - 1, jb = j0 - 1; // grid column / row of the tile's first R1 cell (jb even)
        // 32-bit offsets: creation limits an FP32 jet to 5 fields x fs and its
        // static records to fewer than 2^31 elements
        const int fs = (int)J.fs;
        const int plane = nj * J.pitch;
        const float *__restrict__ Qs = J.q[src];
        float *__restrict__ Qd = J.q[dst];
        const float adt = rhs_only ? 0.0f : c_alpha_f[stage] * (float)dt[jet];
        const float4 *__restrict__ mp = F.mp;
        const long long nrec = (long long)nk * F.njp * 5 * J.pitch;
        (void)nrec; // bound of the static-record checks of a LES_BOUNDS_CHECK build

        // ---- per-item setup ----
        // own column and rows (R1); static-record column and row pair
        const int gi = map_idx(ib + tx, ni, pi);
        const int rA = 2 * tr, rB = 2 * tr + 1;
        const int gjA = map_idx(jb + rA, nj, pj), gjB = map_idx(jb + rB, nj, pj);
        // the two rows share one paired static record (pair jpA) unless a
        // periodic j axis of odd length wraps between them; rows beyond a
        // non-periodic grid read the last record (their values feed no result)
        const bool rec_split = pj && (nj & 1);
        const int jpA = min((pj ? gjA : jb + rA) >> 1, F.njp - 1);
        // in-plane derivative stencils (0: central; +-1: one-sided at a
        // non-periodic end), per column and per row
        const int ti = (!pi && ib + tx == 0) ? 1 : ((!pi && ib + tx == ni - 1) ? -1 : 0);
        const int tjA = (!pj && jb + rA == 0) ? 1 : ((!pj && jb + rA == nj - 1) ? -1 : 0);
        const int tjB = (!pj && jb + rB == nj - 1) ? -1 : 0; // jb even: row 0 is never a second row
        // outputs: columns 1..30, rows 1..TY-2 of R1 inside the output range
        const bool col_out = tx >= 1 && tx <= FX - 2 && (ib + tx) < ihi;
        const bool outA = col_out && rA >= 1 && rA <= TY - 2 && (jb + rA) < jhi;
        const bool outB = col_out && rB >= 1 && rB <= TY - 2 && (jb + rB) < jhi;
        const int ocolA = gjA * J.pitch + gi, ocolB = gjB * J.pitch + gi;
        // slots of the two rows' Q(0) values in QZ (outputs only)
        const int zA = (rA - 1) * (FX - 2) + (tx - 1), zB = (rB - 1) * (FX - 2) + (tx - 1);
        // the R2 pair cells this thread loads (at most two) and, per row, the
        // offset of its source point in the staging box and in a plane
        int lc[2];
        int bo[2][2];
        int go[2][2];
        const CUtensorMap *tmap = nullptr;
        int tx0 = 0;
        if (F.tmap && tma_smem_ok && !pi && !pj && !tma_off) {
            tmap = F.tmap + (TY == 16 ? 3 : 0) + src;
            tx0 = (ib - 1) & ~3;
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = tid + t * NT;
            lc[t] = c < N2 ? c : -1;
            const int cc = (c < N2 ? c : 0) % C2, pr = (c < N2 ? c : 0) / C2;
            const int gc = map_idx(ib - 1 + cc, ni, pi);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gr = map_idx(jb + 2 * (pr - 1) + h, nj, pj);
                go[t][h] = gr * J.pitch + gc;
                int rr = gr - (jb - 2), cl = gc - tx0;
                rr = rr < 0 ? 0 : (rr > BR - 1 ? BR - 1 : rr);
                cl = cl < 0 ? 0 : (cl > TMA_BOX_X - 1 ? TMA_BOX_X - 1 : cl);
                bo[t][h] = rr * TMA_BOX_X + cl;
            }
        }
        if constexpr (SEP) {
            // 1-D spacings of the tile's columns and rows (the previous item's
            // last reads of HX/HY precede its closing barrier)
            if (tid < C2) {
                S.HX[tid] = F.h1[0][map_idx(ib - 1 + tid, ni, pi)];
            } else if (tid < C2 + BR) {
                const int t = tid - C2;
                S.HY[t] = F.h1[1][map_idx(jb - 2 + t, nj, pj)];
            }
        }
        // carried from plane to plane: the zeta flux below, W of the own
        // column one plane below the interface plane, J of the next update
        float2 hz_prev[5], Wc[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            hz_prev[f] = bc(0.0f);
            Wc[f] = bc(0.0f);
        }
        float2 rjU = bc(0.0f), rjG = bc(0.0f);
        __syncthreads(); // shared memory of the previous item is free; HX/HY written

        // thread 0 issues the box of plane kq once every thread is done with
        // the previous one (after a barrier)
        auto stage_box = [&](int kq) {
            if (tid != 0) return;
            const int gk = map_idx(kq, nk, pk);
            tma_box_load(S.QG, tmap, tx0, jb - 2, gk, S.MBAR, G_::BOX_BYTES);
        };
        const int kfirst = k0 - 2, klast = k1 + 1;
        // carried per iteration: grid planes of kL - 2, kL - 1, kL and the
        // three-plane ring slot of kL
        int gkUc = map_idx(kfirst - 2, nk, pk), gkGc = map_idx(kfirst - 1, nk, pk), gkLc = map_idx(kfirst, nk, pk);
        int q3c = r3(kfirst);
        if (tmap) stage_box(kfirst);

        // ---- metric cofactors and J^-1 of grid plane gk for the own row pair
        //      (general form) into MA slot q3: asynchronous copies, waited for one
        //      plane later; where the two rows come from two records, plain loads ----
        auto fetch_met = [&](int gk, int q3) {
            float4 *dst = S.MA + CK_TAB((q3 * 5) * N1 + c1, 15 * N1);
            const int rp = J.pitch;
            if (!rec_split) {
                const int r0 = (gk * F.njp + jpA) * 5 * rp + gi;
                const float4 *p = mp + CK_G(3, r0, nrec);
                (void)CK_G(3, r0 + 4 * rp, nrec);
#pragma unroll
                for (int q = 0; q < 5; ++q) cp_async16(dst + q * N1, p + q * rp);
            } else {
                // rows from two records: take each row's lane
                const int ra = (gk * F.njp + (gjA >> 1)) * 5 * rp + gi;
                const int rb = (gk * F.njp + (gjB >> 1)) * 5 * rp + gi;
                const float4 *pa = mp + CK_G(3, ra, nrec);
                const float4 *pb = mp + CK_G(3, rb, nrec);
                (void)CK_G(3, ra + 4 * rp, nrec);
                (void)CK_G(3, rb + 4 * rp, nrec);
                const bool sa = gjA & 1, sb = gjB & 1;
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const float4 a = pa[q * rp], b = pb[q * rp];
                    dst[q * N1] = make_float4(sa ? a.y : a.x, sb ? b.y : b.x, sa ? a.w : a.z, sb ? b.w : b.z);
                }
            }
        };

        // ---- gradients, closures, sensors, lambda-bar of plane kg (grid plane gk;
        //      three-plane ring slots q3, q3m, q3p of planes kg, kg - 1, kg + 1) ----
        auto grad = [&](int kg, int gk, int q3, int q3m, int q3p) {
            // ring slots of planes kg, kg - 1 (= kg + 2), kg + 1 (= kg - 2)
            const int sl0 = NRING == 4 ? (kg & 3) : q3;
            const int slm = NRING == 4 ? ((kg - 1) & 3) : q3m, slp = NRING == 4 ? ((kg + 1) & 3) : q3p;
            const int slm2 = NRING == 4 ? ((kg - 2) & 3) : q3p, slp2 = NRING == 4 ? ((kg + 2) & 3) : q3m;
            const int s0 = sl0 * N2;
            const int slot = kg & 1;
            const int own = CK_RING(s0 + c2);
            const float4 a0 = S.PA[own], b0 = S.PB[own], q0 = S.PC[own];
            const float2 rho = lo2(a0), p0 = lo2(q0), T0 = hi2(q0);
            const float2 U0[3] = {hi2(a0), lo2(b0), hi2(b0)};
            float2 d[3][4]; // 2 x d/d xi^a of (u, v, w, T)
            float2 nu[3];
            auto sensor = [&](float2 pm, float2 pc, float2 pp) {
                const float2 s = add2(pm, pp);
                const float2 num = fma2(pc, bc(-2.0f), s), den = fma2(pc, bc(2.0f), s);
                const float2 r = rcp2(den);
                return make_float2(fabsf(num.x) * r.x, fabsf(num.y) * r.y);
            };
            // Separable form: derivatives and sensor along xi or zeta in one
            // instruction sequence for every lane, from the cells o1, o2 and the
            // own cell with selected weights: central (t = 0: o1, o2 = c -+ 1,
            // weights 0, -1, 1; sensor over o1, c, o2) or one-sided (o1, o2 =
            // c + t, c + 2t, weights -3t, 4t, -t; sensor over c, o1, o2).  The
            // same values as the branches of the general form below, which keeps
            // the branches (its register budget is tighter; both measured).
            auto axis3 = [&](int o1, int o2, int t, float2 dd[4], float2 &nn) {
                const float4 a1 = S.PA[o1], b1 = S.PB[o1], q1 = S.PC[o1];
                const float4 a2 = S.PA[o2], b2 = S.PB[o2], q2 = S.PC[o2];
                const float tf = (float)t;
                const float2 w0 = bc(-3.0f * tf), w1 = bc(t == 0 ? -1.0f : 4.0f * tf), w2 = bc(t == 0 ? 1.0f : -tf);
                dd[0] = fma2(w2, hi2(a2), fma2(w1, hi2(a1), mul2(w0, U0[0])));
                dd[1] = fma2(w2, lo2(b2), fma2(w1, lo2(b1), mul2(w0, U0[1])));
                dd[2] = fma2(w2, hi2(b2), fma2(w1, hi2(b1), mul2(w0, U0[2])));
                dd[3] = fma2(w2, hi2(q2), fma2(w1, hi2(q1), mul2(w0, T0)));
                nn = sensor(t == 0 ? lo2(q1) : p0, t == 0 ? p0 : lo2(q1), lo2(q2));
            };
            // along xi: central, or one-sided over the cells c, c+t, c+2t at a
            // non-periodic end (the sensor of an end point is its interior
            // neighbour's: same three points)
            if constexpr (SEP) {
                axis3(CK_RING(s0 + c2 + (ti == 0 ? -1 : ti)), CK_RING(s0 + c2 + (ti == 0 ? 1 : 2 * ti)), ti, d[0], nu[0]);
            } else if (ti == 0) {
                const int om = CK_RING(s0 + c2 - 1), op = CK_RING(s0 + c2 + 1);
                const float4 am = S.PA[om], bm = S.PB[om], qm = S.PC[om];
                const float4 ap = S.PA[op], bp = S.PB[op], qp = S.PC[op];
                d[0][0] = sub2(hi2(ap), hi2(am));
                d[0][1] = sub2(lo2(bp), lo2(bm));
                d[0][2] = sub2(hi2(bp), hi2(bm));
                d[0][3] = sub2(hi2(qp), hi2(qm));
                nu[0] = sensor(lo2(qm), p0, lo2(qp));
            } else {
                const int o1 = CK_RING(s0 + c2 + ti), o2 = CK_RING(s0 + c2 + 2 * ti);
                const float4 a1 = S.PA[o1], b1 = S.PB[o1], q1 = S.PC[o1];
                const float4 a2 = S.PA[o2], b2 = S.PB[o2], q2 = S.PC[o2];
                const float2 w0 = bc(-3.0f * ti), w1 = bc(4.0f * ti), w2 = bc(-1.0f * ti);
                d[0][0] = fma2(w2, hi2(a2), fma2(w1, hi2(a1), mul2(w0, U0[0])));
                d[0][1] = fma2(w2, lo2(b2), fma2(w1, lo2(b1), mul2(w0, U0[1])));
                d[0][2] = fma2(w2, hi2(b2), fma2(w1, hi2(b1), mul2(w0, U0[2])));
                d[0][3] = fma2(w2, hi2(q2), fma2(w1, hi2(q1), mul2(w0, T0)));
                nu[0] = sensor(p0, lo2(q1), lo2(q2));
            }
            // along eta: rows 2tr-2 .. 2tr+3 from the pair cells below, own, above
            {
                const int om = CK_RING(s0 + c2 - C2), op = CK_RING(s0 + c2 + C2);
                const float4 am = S.PA[om], bm = S.PB[om], qm = S.PC[om];
                const float4 ap = S.PA[op], bp = S.PB[op], qp = S.PC[op];
                // per field u, v, w, T, p: rows [2tr-2, 2tr-1 | 2tr, 2tr+1 | 2tr+2, 2tr+3]
                const float2 fm[5] = {hi2(am), lo2(bm), hi2(bm), hi2(qm), lo2(qm)};
                const float2 fo[5] = {U0[0], U0[1], U0[2], T0, p0};
                const float2 fp[5] = {hi2(ap), lo2(bp), hi2(bp), hi2(qp), lo2(qp)};
                if (tjA == 0 && tjB == 0) {
#pragma unroll
                    for (int f = 0; f < 4; ++f) d[1][f] = make_float2(fo[f].y - fm[f].y, fp[f].x - fo[f].x);
                    nu[1] = sensor(odd2(fm[4], fo[4]), p0, odd2(fo[4], fp[4]));
                } else {
                    // one row (or both) at an end of a non-periodic j axis:
                    // per row, from the values of rows r-2 .. r+2
                    float v[5][6];
#pragma unroll
                    for (int f = 0; f < 5; ++f) {
                        v[f][0] = fm[f].x; v[f][1] = fm[f].y; v[f][2] = fo[f].x;
                        v[f][3] = fo[f].y; v[f][4] = fp[f].x; v[f][5] = fp[f].y;
                    }
                    float dA[4], dB[4], nA, nB;
                    auto row = [&](int r0, int t, float dd[4], float &nn) {
                        if (t == 0) {
#pragma unroll
                            for (int f = 0; f < 4; ++f) dd[f] = v[f][r0 + 1] - v[f][r0 - 1];
                            const float s = v[4][r0 + 1] + v[4][r0 - 1];
                            nn = fabsf(fmaf(v[4][r0], -2.0f, s)) * __fdividef(1.0f, fmaf(v[4][r0], 2.0f, s));
                        } else {
                            const float w0 = -3.0f * t, w1 = 4.0f * t, w2 = -1.0f * t;
#pragma unroll
                            for (int f = 0; f < 4; ++f)
                                dd[f] = fmaf(w2, v[f][r0 + 2 * t], fmaf(w1, v[f][r0 + t], w0 * v[f][r0]));
                            const float s = v[4][r0] + v[4][r0 + 2 * t];
                            nn = fabsf(fmaf(v[4][r0 + t], -2.0f, s)) * __fdividef(1.0f, fmaf(v[4][r0 + t], 2.0f, s));
                        }
                    };
                    row(2, tjA, dA, nA);
                    row(3, tjB, dB, nB);
#pragma unroll
                    for (int f = 0; f < 4; ++f) d[1][f] = make_float2(dA[f], dB[f]);
                    nu[1] = make_float2(nA, nB);
                }
            }
            // along zeta: the own column one plane below / above, or one-sided
            // at an end of a non-periodic k axis
            {
                const int tk = (!pk && gk == 0) ? 1 : ((!pk && gk == nk - 1) ? -1 : 0);
                if constexpr (SEP) {
                    axis3(CK_RING((tk == 0 ? slm : (tk > 0 ? slp : slm)) * N2 + c2),
                          CK_RING((tk == 0 ? slp : (tk > 0 ? slp2 : slm2)) * N2 + c2), tk, d[2], nu[2]);
                } else if (tk == 0) {
                    const int om = CK_RING(slm * N2 + c2), op = CK_RING(slp * N2 + c2);
                    const float4 am = S.PA[om], bm = S.PB[om], qm = S.PC[om];
                    const float4 ap = S.PA[op], bp = S.PB[op], qp = S.PC[op];
                    d[2][0] = sub2(hi2(ap), hi2(am));
                    d[2][1] = sub2(lo2(bp), lo2(bm));
                    d[2][2] = sub2(hi2(bp), hi2(bm));
                    d[2][3] = sub2(hi2(qp), hi2(qm));
                    nu[2] = sensor(lo2(qm), p0, lo2(qp));
                } else {
                    const int o1 = CK_RING((tk > 0 ? slp : slm) * N2 + c2), o2 = CK_RING((tk > 0 ? slp2 : slm2) * N2 + c2);
                    const float4 a1 = S.PA[o1], b1 = S.PB[o1], q1 = S.PC[o1];
                    const float4 a2 = S.PA[o2], b2 = S.PB[o2], q2 = S.PC[o2];
                    const float2 w0 = bc(-3.0f * tk), w1 = bc(4.0f * tk), w2 = bc(-1.0f * tk);
                    d[2][0] = fma2(w2, hi2(a2), fma2(w1, hi2(a1), mul2(w0, U0[0])));
                    d[2][1] = fma2(w2, lo2(b2), fma2(w1, lo2(b1), mul2(w0, U0[1])));
                    d[2][2] = fma2(w2, hi2(b2), fma2(w1, hi2(b1), mul2(w0, U0[2])));
                    d[2][3] = fma2(w2, hi2(q2), fma2(w1, hi2(q1), mul2(w0, T0)));
                    nu[2] = sensor(p0, lo2(q1), lo2(q2));
                }
            }
            // metrics: cofactors m (rows of d xi^a / d x times J^-1), J,
            // (Cs Delta)^2 J, row norms
            float2 m[9], rj, csdJ, nrm[3], rh[3];
            if constexpr (SEP) {
                // diagonal cofactors: 1/h_a per axis; J = prod 1/h_a
                const float4 hX = S.HX[tx + 1];
                const float4 hYA = S.HY[rA + 2], hYB = S.HY[rB + 2];
                const float4 hZ = S.HZ[kg & 3];
                rh[0] = bc(hX.y);
                rh[1] = f2(hYA.y, hYB.y);
                rh[2] = bc(hZ.y);
                csdJ = mul2(bc(FP.cs2 * hX.z * hZ.z), f2(hYA.z, hYB.z)); // (Cs Delta)^2, Delta^3 = h_x h_y h_z
                rj = mul2(bc(hX.y * hZ.y), rh[1]);
#pragma unroll
                for (int t = 0; t < 9; ++t) m[t] = bc(0.0f);
#pragma unroll
                for (int a = 0; a < 3; ++a) nrm[a] = bc(0.0f);
            } else {
                float4 u[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) u[q] = S.MA[CK_TAB((q3 * 5 + q) * N1 + c1, 15 * N1)];
                m[0] = lo2(u[0]); m[1] = hi2(u[0]); m[2] = lo2(u[1]); m[3] = hi2(u[1]);
                m[4] = lo2(u[2]); m[5] = hi2(u[2]); m[6] = lo2(u[3]); m[7] = hi2(u[3]);
                m[8] = lo2(u[4]);
                // J, (Cs Delta)^2 J = Cs^2 (J^-1)^(-1/3) with Delta = (J^-1)^(1/3), and
                // the row norms |grad xi^a| / J; on the degenerate axis of a polar
                // mesh (J^-1 = 0) J = 1 and the filter width is zero
                const float2 jv = hi2(u[4]);
                rj = make_float2(jv.x > 0.0f ? __fdividef(1.0f, jv.x) : 1.0f, jv.y > 0.0f ? __fdividef(1.0f, jv.y) : 1.0f);
                csdJ = make_float2(jv.x > 0.0f ? FP.cs2 * rcbrtf(jv.x) : 0.0f, jv.y > 0.0f ? FP.cs2 * rcbrtf(jv.y) : 0.0f);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    nrm[a] = sqrt2(fma2(m[3 * a + 2], m[3 * a + 2], fma2(m[3 * a + 1], m[3 * a + 1], mul2(m[3 * a], m[3 * a]))));
                    rh[a] = bc(0.0f);
                }
            }
            // doubled physical velocity gradient g' (2 J^-1 du_i/dx_c for the
            // general form, 2 du_i/dx_c separable), strain norm, Smagorinsky
            float2 g[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    if constexpr (SEP) g[i][cc] = mul2(d[cc][i], rh[cc]);
                    else g[i][cc] = fma2(m[6 + cc], d[2][i], fma2(m[3 + cc], d[1][i], mul2(m[cc], d[0][i])));
                }
            const float2 a01 = add2(g[0][1], g[1][0]), a02 = add2(g[0][2], g[2][0]), a12 = add2(g[1][2], g[2][1]);
            const float2 sd = fma2(g[2][2], g[2][2], fma2(g[1][1], g[1][1], mul2(g[0][0], g[0][0])));
            const float2 so = fma2(a12, a12, fma2(a02, a02, mul2(a01, a01)));
            // |S| = (2 S_ij S_ij)^1/2 = J sqrt(sd/2 + so/4) in terms of g'
            const float2 mus = mul2(mul2(rho, csdJ), sqrt2(fma2(so, bc(0.25f), mul2(sd, bc(0.5f)))));
            // Sutherland mu(T), speed of sound c = T^1/2
            const float2 sT = sqrt2(T0);
            const float2 mu = mul2(mul2(T0, sT), mul2(bc(FP.suth1), rcp2(add2(T0, bc(FP.suthS)))));
            const float2 mue = fma2(mu, bc(FP.inv_Re), mus);
            const float2 kap = fma2(mu, bc(FP.kap_mol), mul2(mus, bc(FP.kap_sgs)));
            // spectral radii lambda_a = |U_a| + c |grad xi^a|, lambda-bar_a =
            // s_a (s_a + s_b + s_d) with s = lambda^1/2
            float2 sq[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float2 lam;
                if constexpr (SEP) {
                    const float2 ua = U0[a];
                    lam = mul2(make_float2(fabsf(ua.x) + sT.x, fabsf(ua.y) + sT.y), rh[a]);
                } else {
                    const float2 JU = fma2(m[3 * a + 2], U0[2], fma2(m[3 * a + 1], U0[1], mul2(m[3 * a], U0[0])));
                    lam = mul2(make_float2(fmaf(sT.x, nrm[a].x, fabsf(JU.x)), fmaf(sT.y, nrm[a].y, fabsf(JU.y))),
                               rj);
                }
                sq[a] = sqrt2(lam);
            }
            const float2 ssum = add2(add2(sq[0], sq[1]), sq[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                S.GD[CK_TAB((slot * 6 + 2 * a) * N1 + c1, 12 * N1)] = cat4(d[a][0], d[a][1]);
                S.GD[CK_TAB((slot * 6 + 2 * a + 1) * N1 + c1, 12 * N1)] = cat4(d[a][2], d[a][3]);
            }
            S.GC[CK_TAB((slot * 4) * N1 + c1, 8 * N1)] = cat4(mue, kap);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                S.GC[CK_TAB((slot * 4 + 1 + a) * N1 + c1, 8 * N1)] = cat4(nu[a], mul2(sq[a], ssum));
            rjG = rj;
        };

        // ---- shared-memory accessors of the interface phase ----
        auto pts = [&](int cell) {
            Pts P;
            const float4 a = S.PA[cell], b = S.PB[cell], q = S.PC[cell];
            P.rho = lo2(a); P.u = hi2(a); P.v = lo2(b); P.w = hi2(b); P.p = lo2(q); P.T = hi2(q);
            P.rH = S.PH[cell];
            return P;
        };
        auto wof = [&](int cell, float2 W[5]) {
            const float4 a = S.PA[cell], b = S.PB[cell];
            const float2 rho = lo2(a);
            W[0] = rho;
            W[1] = mul2(rho, hi2(a));
            W[2] = mul2(rho, lo2(b));
            W[3] = mul2(rho, hi2(b));
            W[4] = S.PH[cell];
        };
        auto mets = [&](int slot, int cell, float2 m[9], float2 &jv) {
            float4 u[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) u[q] = S.MA[CK_TAB((slot * 5 + q) * N1 + cell, 15 * N1)];
            m[0] = lo2(u[0]); m[1] = hi2(u[0]); m[2] = lo2(u[1]); m[3] = hi2(u[1]);
            m[4] = lo2(u[2]); m[5] = hi2(u[2]); m[6] = lo2(u[3]); m[7] = hi2(u[3]);
            m[8] = lo2(u[4]);
            jv = hi2(u[4]);
        };
        // transport data along axis A: coefficients, (nu_A, lb_A), and
        // the doubled derivatives along the two other axes
        auto side = [&](int A, int slot, int cell, Side &Sd) {
            const float4 c0 = S.GC[CK_TAB((slot * 4) * N1 + cell, 8 * N1)];
            const float4 ca = S.GC[CK_TAB((slot * 4 + 1 + A) * N1 + cell, 8 * N1)];
            Sd.mue = lo2(c0); Sd.kap = hi2(c0); Sd.nu = lo2(ca); Sd.lb = hi2(ca);
            const int b1 = A == 0 ? 1 : 0, b2 = A == 2 ? 1 : 2;
            const float4 e0 = S.GD[CK_TAB((slot * 6 + 2 * b1) * N1 + cell, 12 * N1)];
            const float4 e1 = S.GD[CK_TAB((slot * 6 + 2 * b1 + 1) * N1 + cell, 12 * N1)];
            const float4 f0 = S.GD[CK_TAB((slot * 6 + 2 * b2) * N1 + cell, 12 * N1)];
            const float4 f1v = S.GD[CK_TAB((slot * 6 + 2 * b2 + 1) * N1 + cell, 12 * N1)];
            Sd.d[0][0] = lo2(e0); Sd.d[0][1] = hi2(e0); Sd.d[0][2] = lo2(e1); Sd.d[0][3] = hi2(e1);
            Sd.d[1][0] = lo2(f0); Sd.d[1][1] = hi2(f0); Sd.d[1][2] = lo2(f1v); Sd.d[1][3] = hi2(f1v);
        };
        for (int kL = kfirst; kL <= klast; ++kL) {
            const int kG = kL - 1, kU = kL - 2;
            // slots of planes kL, kG, kU in the three-plane rings, and their
            // grid planes
            const int q3L = q3c, q3G = q3L == 0 ? 2 : q3L - 1, q3U = q3L == 2 ? 0 : q3L + 1;
            const int gkLm = gkLc, gkGm = gkGc, gkUm = gkUc;
            const int sLr = NRING == 4 ? (kL & 3) : q3L, sGr = NRING == 4 ? (kG & 3) : q3G, sUr = NRING == 4 ? (kU & 3) : q3U;
            const bool do_grad = kG >= k0 - 1 && kG <= k1 && !(!pk && kG == 0);
            // the first plane of a non-periodic k axis: formed with plane 1
            const bool do_grad0 = !pk && kG == 1 && k0 == 1;
            // the mirror plane beyond the last plane of a non-periodic k axis is
            // not loaded (its slot still holds a plane the last gradients need);
            // the last interface takes the mirror from its own plane
            const bool ghost_hi = !pk && kL == nk;
            // ---- load + primitives of plane kL on R2 ----
            if (!ghost_hi) {
                const int gkL = gkLm;
                bool from_box = false;
                if (tmap) {
                    // the box of this plane (issued one iteration earlier); a
                    // wait that gives up is recorded (site 8) instead of
                    // hanging, and this thread reads the plane from global memory
                    if (mbar_wait(S.MBAR, tpar, wait_limit)) {
                        from_box = true;
                        tpar ^= 1u;
                    } else {
                        if (J.oob) atomicCAS(J.oob, 0ull, 8ull << 48);
                        tma_off = true;
                        pend = true;
                    }
                }
                const int sb = sLr * N2;
                const int pofs = gkL * plane;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (lc[t] < 0) continue;
                    float q[2][5];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (from_box) {
#pragma unroll
                            for (int f = 0; f < 5; ++f)
                                q[h][f] = S.QG[CK_TAB(f * (BR * TMA_BOX_X) + bo[t][h], 5 * BR * TMA_BOX_X)];
                        } else {
                            const int o = CK_G(2, pofs + go[t][h], J.npts_pad);
#pragma unroll
                            for (int f = 0; f < 5; ++f) q[h][f] = Qs[f * fs + o];
                        }
                    }
                    const float2 rho = f2(q[0][0], q[1][0]);
                    const float2 rr = rcp2(rho);
                    const float2 u = mul2(f2(q[0][1], q[1][1]), rr), v = mul2(f2(q[0][2], q[1][2]), rr),
                                 ww = mul2(f2(q[0][3], q[1][3]), rr);
                    const float2 e = f2(q[0][4], q[1][4]);
                    const float2 q2 = fma2(ww, ww, fma2(v, v, mul2(u, u)));
                    const float2 p = mul2(bc(FP.gm1), fma2(mul2(rho, q2), bc(-0.5f), e));
                    const int cell = CK_RING(sb + lc[t]);
                    S.PA[cell] = cat4(rho, u);
                    S.PB[cell] = cat4(v, ww);
                    S.PC[cell] = cat4(p, mul2(mul2(bc(FP.gam), p), rr));
                    S.PH[cell] = add2(e, p);
                }
            }
            // separable form: thread 0's spacing copy of plane kL - 1 (issued
            // two iterations ago) has landed, and the barrier publishes it
            if (SEP && tid == 0) cp_async_wait_prev();
            // (a thread whose staging wait gave up turns staging off for the
            // whole CTA here)
            tma_off = __syncthreads_or(tma_off) != 0;
            if (tma_off) tmap = nullptr;
            // the next plane's box, in flight during the rest of this iteration
            if (tmap && kL < klast && !(!pk && kL + 1 == nk)) stage_box(kL + 1);
            // one copy group per iteration: the metrics of the next gradient
            // plane (kL), waited for in the next iteration, and Q(0) of this
            // iteration's updated points (plane kL - 2), waited for before
            // the update; each thread copies, and later reads, its own values
            if constexpr (!SEP) {
                if (kL >= k0 - 1 && kL <= k1) fetch_met(gkLm, q3L);
            } else {
                // the spacings of plane kL + 1 into the slot of plane kL - 3,
                // whose last reads preceded the barrier above
                if (tid == 0) cp_async16(S.HZ + ((kL + 1) & 3), F.h1[2] + map_idx(kL + 1, nk, pk));
            }
            if (!rhs_only && kL - 2 >= k0 && kL - 2 <= k1 - 1) {
                const int pU = gkUm * plane;
                const float *Q0 = J.q[0];
                if (outA) {
                    const int oA = CK_G(4, pU + ocolA, J.npts_pad);
#pragma unroll
                    for (int f = 0; f < 5; ++f) cp_async4(S.QZ + CK_TAB(f * G_::QZN + zA, 5 * G_::QZN), Q0 + f * fs + oA);
                }
                if (outB) {
                    const int oB = CK_G(4, pU + ocolB, J.npts_pad);
#pragma unroll
                    for (int f = 0; f < 5; ++f) cp_async4(S.QZ + CK_TAB(f * G_::QZN + zB, 5 * G_::QZN), Q0 + f * fs + oB);
                }
            }
            cp_async_commit();
            // W of the own column at plane k0 - 2: the outer point of the
            // chunk's first zeta interface
            if (kL == k0) wof(CK_RING(sUr * N2 + c2), Wc);
            // ---- gradients of plane kG (and of plane 0, late) ----
            if (!SEP && (do_grad || do_grad0)) cp_async_wait_prev();
            if (do_grad0) grad(0, map_idx(0, nk, pk), r3(0), r3(-1), r3(1));
            if (do_grad) grad(kG, gkGm, q3G, q3U, q3L);
            // ---- interfaces and update of plane kU ----
            if (kU >= k0 - 1 && kU <= k1 - 1) {
                const bool first = kU == k0 - 1; // only the -1/2 zeta flux of the chunk
                const int gkU = gkUm;
                const int sU = sUr * N2, sUp = sGr * N2, sUpp = sLr * N2;
                const int rU = (kU & 1), rP = ((kU + 1) & 1); // R1 tables
                const int mU = q3U, mP = q3G;       // metric tables
                // own points at plane kU
                const Pts L = pts(CK_RING(sU + c2));
                float2 WL[5];
                wvec(L, WL);
                float2 mL[9], jL = bc(0.0f);
                if constexpr (!SEP) mets(mU, c1, mL, jL);
                // separable form: spacings of the own points and their neighbours
                float4 hXo = make_float4(0.f, 0.f, 0.f, 0.f), hXp = hXo, hZo = hXo, hZp = hXo;
                float2 hYo = bc(0.f), rhYo = bc(0.f);
                if constexpr (SEP) {
                    hXo = S.HX[tx + 1];
                    hXp = S.HX[tx + 2];
                    hZo = S.HZ[kU & 3];
                    hZp = S.HZ[(kU + 1) & 3];
                    const float4 yA = S.HY[rA + 2], yB = S.HY[rB + 2];
                    hYo = f2(yA.x, yB.x);
                    rhYo = f2(yA.y, yB.y);
                }
                float2 hx[5], hy[5], hz[5];
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    hx[f] = bc(0.0f);
                    hy[f] = bc(0.0f);
                    hz[f] = bc(0.0f);
                }
                const bool updA = !first && outA && kU >= k0, updB = !first && outB && kU >= k0;
                const int pU = gkU * plane;
                const int oA = CK_G(4, pU + ocolA, J.npts_pad), oB = CK_G(4, pU + ocolB, J.npts_pad);
                // zeta: R = the own column one plane up; R + 1 two planes up;
                // L - 1 one plane down (carried, or read on the first plane).
                // General form: evaluated between the eta and the xi flux in one
                // block (independent work for the scheduler to interleave; of the
                // orders measured, eta-zeta-xi ran fastest)
                auto zeta = [&]() {
                    const Pts R = pts(CK_RING(sUp + c2));
                    float2 WR[5], WRp[5];
                    wvec(R, WR);
                    if (ghost_hi) {
#pragma unroll
                        for (int f = 0; f < 5; ++f) WRp[f] = WL[f]; // W(nk) = W(nk - 2)
                    } else {
                        wof(CK_RING(sUpp + c2), WRp);
                    }
                    Side SL, SR;
                    side(2, rU, c1, SL);
                    side(2, rP, c1, SR);
                    if constexpr (SEP) {
                        const float2 Sa = mul2(bc(hXo.x), hYo);
                        const float2 hb = bc(0.5f * (hZo.x + hZp.x));
                        iface_sep<2>(FP, L, WL, R, WR, Wc, WRp, SL, SR, Sa, hb, rcp2(hb), bc(0.25f * hXo.y),
                                     mul2(bc(0.25f), rhYo), hz);
                    } else {
                        float2 mR[9], jR;
                        mets(mP, c1, mR, jR);
                        iface<2>(FP, L, WL, mL, jL, R, WR, mR, jR, Wc, WRp, SL, SR, hz);
                    }
                };
                if (!first) {
                    // eta: R = (own second row, first row of the pair cell
                    // above); R + 1 = the pair cell above; L - 1 = (second row
                    // of the pair cell below, own first row)
                    {
                        const int up = tr + 1 < TR ? c1 + FX : c1; // the top thread row's second flux is not used
                        const Pts P1 = pts(CK_RING(sU + c2 + C2));
                        const Pts R = odd_pts(L, P1);
                        float2 WP1[5], WR[5], WLm[5], Wm[5];
                        wvec(P1, WP1);
                        wof(CK_RING(sU + c2 - C2), Wm);
#pragma unroll
                        for (int f = 0; f < 5; ++f) {
                            WR[f] = odd2(WL[f], WP1[f]);
                            WLm[f] = odd2(Wm[f], WL[f]);
                        }
                        Side SL, SU, SR;
                        side(1, rU, c1, SL);
                        side(1, rU, up, SU);
                        SR.mue = odd2(SL.mue, SU.mue);
                        SR.kap = odd2(SL.kap, SU.kap);
                        SR.nu = odd2(SL.nu, SU.nu);
                        SR.lb = odd2(SL.lb, SU.lb);
#pragma unroll
                        for (int b = 0; b < 2; ++b)
#pragma unroll
                            for (int f = 0; f < 4; ++f) SR.d[b][f] = odd2(SL.d[b][f], SU.d[b][f]);
                        if constexpr (SEP) {
                            const float4 yC = S.HY[rB + 3]; // row 2tr+2
                            const float2 hYR = f2(hYo.y, yC.x);
                            const float2 Sa = bc(hXo.x * hZo.x);
                            const float2 hb = mul2(bc(0.5f), add2(hYo, hYR));
                            iface_sep<1>(FP, L, WL, R, WR, WLm, WP1, SL, SR, Sa, hb, rcp2(hb), bc(0.25f * hXo.y),
                                         bc(0.25f * hZo.y), hy);
                        } else {
                            float2 mA[9], jA, mR[9];
                            mets(mU, up, mA, jA);
#pragma unroll
                            for (int t = 0; t < 9; ++t) mR[t] = odd2(mL[t], mA[t]);
                            iface<1>(FP, L, WL, mL, jL, R, WR, mR, odd2(jL, jA), WLm, WP1, SL, SR, hy);
                        }
                    }
                    if constexpr (!SEP) zeta();
                    // xi: R = the next column.  Lane 31's R has no R1 data: it pairs
                    // with its own R1 cell (an unused result), so that every lane
                    // runs the xi flux without a branch and the scheduler can
                    // interleave it with the eta flux
                    {
                        const int cR = tx <= FX - 2 ? c1 + 1 : c1;
                        const Pts R = pts(CK_RING(sU + c2 + 1));
                        float2 WR[5], WRp[5], WLm[5];
                        wvec(R, WR);
                        wof(CK_RING(sU + c2 + 2), WRp);
                        wof(CK_RING(sU + c2 - 1), WLm);
                        Side SL, SR;
                        side(0, rU, c1, SL);
                        side(0, rU, cR, SR);
                        if constexpr (SEP) {
                            // Sa = h_y h_z, hb = average h_x, tangential 1/(4 h)
                            const float2 Sa = mul2(hYo, bc(hZo.x));
                            const float2 hb = bc(0.5f * (hXo.x + hXp.x));
                            iface_sep<0>(FP, L, WL, R, WR, WLm, WRp, SL, SR, Sa, hb, rcp2(hb),
                                         mul2(bc(0.25f), rhYo), bc(0.25f * hZo.y), hx);
                        } else {
                            float2 mR[9], jR;
                            mets(mU, cR, mR, jR);
                            iface<0>(FP, L, WL, mL, jL, R, WR, mR, jR, WLm, WRp, SL, SR, hx);
                        }
                    }
#pragma unroll
                    for (int f = 0; f < 5; ++f) S.SH[CK_SH(f * NT + tid)] = hy[f].y;
                } else if constexpr (!SEP) {
                    zeta();
                }
                if constexpr (SEP) zeta();
                // the -1/2 xi flux from the lane below (all lanes of the warp
                // take part in the shuffle; the CTA-uniform `first` guards it)
                float2 hxm[5];
#pragma unroll
                for (int f = 0; f < 5; ++f) hxm[f] = bc(0.0f);
                if (!first) {
#pragma unroll
                    for (int f = 0; f < 5; ++f)
                        hxm[f] = f2(__shfl_up_sync(0xffffffffu, hx[f].x, 1), __shfl_up_sync(0xffffffffu, hx[f].y, 1));
                }
                __syncthreads(); // eta fluxes of the row below; the first plane's read of W below
                if (updA || updB) {
                    cp_async_wait_all(); // this thread's Q(0) copies
                    // residual R = sum over axes of flux(+1/2) - flux(-1/2); the
                    // -1/2 zeta flux from the previous plane, the -1/2 eta flux
                    // of the first row from the thread row below and of the
                    // second row from the own first
                    float2 Rs[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f) {
                        const float hyb = tr > 0 ? S.SH[CK_SH(f * NT + tid - FX)] : 0.0f;
                        const float2 hym = f2(hyb, hy[f].x);
                        Rs[f] = add2(add2(sub2(hx[f], hxm[f]), sub2(hy[f], hym)), sub2(hz[f], hz_prev[f]));
                    }
                    if (rhs_only) {
                        if (updA) {
#pragma unroll
                            for (int f = 0; f < 5; ++f) J.rhs[f * fs + oA] = Rs[f].x;
                        }
                        if (updB) {
#pragma unroll
                            for (int f = 0; f < 5; ++f) J.rhs[f * fs + oB] = Rs[f].y;
                        }
                    } else {
                        // the stored state is unscaled: Q(l) = Q(0) - alpha dt J RHS
                        const float2 adtj = mul2(bc(adt), rjU);
                        if (updA) {
#pragma unroll
                            for (int f = 0; f < 5; ++f)
                                Qd[f * fs + oA] = fmaf(-adtj.x, Rs[f].x, S.QZ[CK_TAB(f * G_::QZN + zA, 5 * G_::QZN)]);
                        }
                        if (updB) {
#pragma unroll
                            for (int f = 0; f < 5; ++f)
                                Qd[f * fs + oB] = fmaf(-adtj.y, Rs[f].y, S.QZ[CK_TAB(f * G_::QZN + zB, 5 * G_::QZN)]);
                        }
                    }
                }
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    hz_prev[f] = hz[f];
                    Wc[f] = WL[f];
                }
            } else if (NRING == 3) {
                __syncthreads(); // as in the branch above: this iteration's ring reads
                                 // precede the next iteration's loads into the freed slot
            }
            rjU = rjG; // plane kG is the next iteration's kU
            gkUc = gkGc;
            gkGc = gkLc;
            gkLc = map_idx(kL + 1, nk, pk);
            q3c = q3U;
        }
    }
    cp_async_wait_all();
    // a copy whose wait gave up may still be in flight into this CTA's
    // shared memory: its issuer waits for it (bounded) before exiting; if
    // that wait gives up too, the copy may land in the shared memory of the
    // next CTA on this SM, which is recorded as site 9 (it outranks site 8:
    // the state can no longer be trusted)
    if (pend && tid == 0 && !mbar_wait(S.MBAR, tpar, MBAR_WAIT_LIMIT)) {
        const JetDev<float> &J0 = jet_entry<ONE>(j1, jets, 0);
        if (J0.oob) atomicMax(J0.oob, 9ull << 48);
    }
}

#undef CK_G
#undef CK_RING
#undef CK_TAB
#undef CK_SH

// Paired static records of the general FP32 form (see FusedJet::mp).  The
// padding row of an odd nj is zero.
__global__ void __launch_bounds__(BLOCK) k_pack_pairs(const float *__restrict__ met, long long fs, int pitch,
                                                      int nj, int nk, float4 *__restrict__ mp)
{
    const int njp = (nj + 1) / 2;
    const long long total = (long long)nk * njp * pitch;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % pitch);
        const long long r = t / pitch;
        const int jp = (int)(r % njp), k = (int)(r / njp);
        float v[2][10];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * jp + h;
#pragma unroll
            for (int c = 0; c < 10; ++c) v[h][c] = 0.0f;
            if (j >= nj) continue;
            const float *m = met + ((long long)k * nj + j) * pitch + i;
#pragma unroll
            for (int c = 0; c < 9; ++c) v[h][c] = m[c * fs];
            v[h][9] = m[MET_JINV * fs];
        }
        float4 *out = mp + (r * 5) * pitch + i;
#pragma unroll
        for (int q = 0; q < 5; ++q)
            out[q * pitch] = make_float4(v[0][2 * q], v[1][2 * q], v[0][2 * q + 1], v[1][2 * q + 1]);
    }
}

void launch_pack_pairs(const float *met, long long fs, int pitch, int nj, int nk, float4 *mp, cudaStream_t st)
{
    const long long total = (long long)nk * ((nj + 1) / 2) * pitch;
    k_pack_pairs<<<(int)std::min<long long>((total + BLOCK - 1) / BLOCK, 65535LL * 4), BLOCK, 0, st>>>(
        met, fs, pitch, nj, nk, mp);
}

template <int TY> int fused_prepare()
{
    int rc = (int)cudaFuncSetAttribute(k_fused<TY, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Geo<TY, false>::BYTES);
    if (!rc) rc = (int)cudaFuncSetAttribute(k_fused<TY, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)Geo<TY, true>::BYTES);
    if (!rc) rc = (int)cudaFuncSetAttribute(k_fused<TY, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)Geo<TY, false>::BYTES);
    if (!rc) rc = (int)cudaFuncSetAttribute(k_fused<TY, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)Geo<TY, true>::BYTES);
    return rc;
}

int fused_ctas_per_sm(int ty, int separable)
{
    int n = 0;
    cudaError_t e;
    if (ty == 16)
        e = separable ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<16, true, true>, FX * 8,
                                                                      Geo<16, true>::BYTES)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<16, false, true>, FX * 8,
                                                                      Geo<16, false>::BYTES);
    else
        e = separable ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<8, true, true>, FX * 4,
                                                                      Geo<8, true>::BYTES)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<8, false, true>, FX * 4,
                                                                      Geo<8, false>::BYTES);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <int TY>
void launch_fused(const JetDev<float> *jets, const FusedJet *fj, int njets, int total_items, int total_tiles,
                  int grid, int src, int dst, int stage, const double *dt, int rhs_only, int separable, int balanced,
                  int wait_limit, const JetDev<float> *j1, const FusedJet *f1, cudaStream_t st)
{
    dim3 block(FX, TY / 2);
    if (wait_limit < 0) wait_limit = MBAR_WAIT_LIMIT;
    const bool one = njets == 1 && j1 && f1;
    JetDev<float> jz{};
    FusedJet fz{};
    const JetDev<float> &ja = one ? *j1 : jz;
    const FusedJet &fa = one ? *f1 : fz;
    if (separable) {
        if (one)
            k_fused<TY, true, true><<<grid, block, Geo<TY, true>::BYTES, st>>>(
                jets, fj, njets, total_items, total_tiles, src, dst, stage, dt, rhs_only, balanced, wait_limit, ja, fa);
        else
            k_fused<TY, true, false><<<grid, block, Geo<TY, true>::BYTES, st>>>(
                jets, fj, njets, total_items, total_tiles, src, dst, stage, dt, rhs_only, balanced, wait_limit, ja, fa);
    } else {
        if (one)
            k_fused<TY, false, true><<<grid, block, Geo<TY, false>::BYTES, st>>>(
                jets, fj, njets, total_items, total_tiles, src, dst, stage, dt, rhs_only, balanced, wait_limit, ja, fa);
        else
            k_fused<TY, false, false><<<grid, block, Geo<TY, false>::BYTES, st>>>(
                jets, fj, njets, total_items, total_tiles, src, dst, stage, dt, rhs_only, balanced, wait_limit, ja, fa);
    }
}

template int fused_prepare<16>();
template int fused_prepare<8>();
template void launch_fused<16>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int, int,
                               const double *, int, int, int, int, const JetDev<float> *, const FusedJet *,
                               cudaStream_t);
template void launch_fused<8>(const JetDev<float> *, const FusedJet *, int, int, int, int, int, int, int,
                              const double *, int, int, int, int, const JetDev<float> *, const FusedJet *,
                              cudaStream_t);

} // namespace les
