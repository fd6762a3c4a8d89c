// tp_pair.cu -- the particle-particle force loop (Sec. II-A; "force
// calculation" in Table I) and its adjoint.
//
// Work unit: one group and its interaction list.  A CTA stages list entries as
// group-relative offsets in shared memory (tiles of kTile) and each thread
// keeps one i-particle in registers; when the group is smaller than the CTA,
// several threads hold the same i and split the list between them ("streams"),
// and their partial sums are reduced at the end in a fixed order.
//
// Group-relative offsets come from the 64-bit fixed-point images: the
// wrap-around integer difference of two images is the exact periodic minimum
// image offset, so the only rounding is the final conversion to the working
// precision.  Offsets are scaled by k = 2/r_cut, so the cutoff argument of
// Eq. 3 is xi = |d'| and the cutoff test is |d'|^2 < 4; the sum is multiplied
// by G k^2 once per particle.
#include "tp_common.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;
// Tile shapes (chosen per tree, see tp_tree_set_tile): particles per thread of
// the forward pair kernel (1, 2 or 4) and list entries per thread of the fused
// adjoint (2 or 4).

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The MUFU reciprocal square root without denormal handling.  The packed pair
// kernels take it of s'^2 = |d'|^2 + (k eps)^2 >= (k eps)^2 > 0, always a
// normal number; rsqrtf() would wrap the same MUFU operation in a test and two
// scalar multiplies for denormal inputs (measured: 4 extra FMA-pipe cycles per
// packed pair step, about 6 % of the forward kernel's FMA-pipe work).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (two lanes of one 64-bit register): Blackwell executes
// add/sub/mul/fma.f32x2 as one instruction, halving the issue slots of the
// pair arithmetic.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 f2relu(f2 v)
{
    float a, b;
    f2unpack(v, a, b);
    return f2pack(fmaxf(a, 0.f), fmaxf(b, 0.f));
}

// The paper's inverse square root (Sec. II-A), a kernel variant
// (TP_FLAG_RSQRT_REFINED) that takes 1/s' off the MUFU pipe: an estimate y0
// refined by one third-order step, h0 = 1 - x y0^2, y1 = y0 (1 + h0/2 +
// 3 h0^2/8), relative error 5/2 e^3 + O(e^4) for an estimate off by e.  The
// K computer's estimate instruction gives 8 bits; the estimate here is the
// integer approximation of Lomont (2003): the bit pattern of x shifted right
// by one and subtracted from 0x5f3759df (|e| < 3.5e-2), then one Newton step
// y (3/2 - x y^2/2) (|e| < 1.8e-3), so y1 is good to ~1.5e-8.  Ten packed
// FP32 operations and two integer ones per pair of roots, for x > 0 normal.
__device__ __forceinline__ f2 rsqrt_refined(f2 x)
{
    float xa, xb;
    f2unpack(x, xa, xb);
    const f2 y0 = f2pack(__uint_as_float(0x5f3759dfu - (__float_as_uint(xa) >> 1)),
                         __uint_as_float(0x5f3759dfu - (__float_as_uint(xb) >> 1)));
    const f2 nx = f2mul(x, f2pack(-1.f, -1.f));
    const f2 nhx = f2mul(x, f2pack(-0.5f, -0.5f));
    const f2 y = f2mul(y0, f2fma(nhx, f2mul(y0, y0), f2pack(1.5f, 1.5f)));
    const f2 h0 = f2fma(nx, f2mul(y, y), f2pack(1.f, 1.f));
    const f2 p = f2fma(f2pack(0.375f, 0.375f), h0, f2pack(0.5f, 0.5f));
    return f2fma(f2mul(y, h0), p, y);
}

template <class R> struct Arith;

template <> struct Arith<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrt_approx(x); }
    // sqrt(s2) on the MUFU pipe, which has room to spare in these kernels;
    // s2 * rsqrt(s2) would save the MUFU op but add an FMUL on the FMA pipe,
    // the one that bounds them (measured 1-3 % slower)
    static __device__ __forceinline__ float soft_xi(float s2, float) { return sqrt_approx(s2); }
    static __device__ __forceinline__ float from_fixed(uint64_t a, uint64_t b, float sc)
    {
        return tp_offset_f32(a, b, sc);
    }
};

template <> struct Arith<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double soft_xi(double s2, double) { return ::sqrt(s2); }
    static __device__ __forceinline__ double from_fixed(uint64_t a, uint64_t b, double sc)
    {
        return __ll2double_rn((long long)(a - b)) * sc;
    }
};

// Eq. 3 evaluated branch by branch.  The paper's branch-free nested form
// (with the zeta = max(0, xi - 1) correction) is exact in FP64, but in FP32 its
// O(1) terms cancel to O(1e-6) near xi = 2 (20 % relative error at xi = 1.9).
// Here the interval [0,1] uses the expanded polynomial of Eq. 3 and [1,2] the
// same polynomial factored as (2 - xi)^5 (7 xi^3 + 22 xi^2 + 10 xi + 4) / 140,
// whose relative error stays at a few FP32 ulps all the way to the cutoff; the
// two are selected per pair (both are evaluated, no divergence).
template <class R>
__device__ __forceinline__ R g_p3m(R xi, R r2)
{
    R p = R(3.0 / 20.0) * xi + R(-12.0 / 35.0);
    p = p * xi + R(-0.5);
    p = p * xi + R(8.0 / 5.0);
    p = p * r2 + R(-8.0 / 5.0);
    const R lo = p * (r2 * xi) + R(1.0);
    const R u = R(2.0) - xi;
    R h = R(7.0 / 140.0) * xi + R(22.0 / 140.0);
    h = h * xi + R(10.0 / 140.0);
    h = h * xi + R(4.0 / 140.0);
    const R u2 = u * u;
    const R hi = (u2 * u2 * u) * h;
    return xi <= R(1.0) ? lo : hi;
}

struct Group {
    int32_t first, ni;
    int64_t e0;
    int32_t ne;
    uint64_t X, Y, Z;
    const BoxPrm *P;
    bool wrap;   // offsets of i and j may differ by more than half a box
};

__device__ __forceinline__ Group load_group(const TreeDev &T, int64_t g)
{
    Group G;
    G.first = T.gfirst[g];
    G.ni = T.gcount[g];
    G.e0 = T.loff[g];
    G.ne = T.lcnt[g];
    G.X = T.gX[g]; G.Y = T.gY[g]; G.Z = T.gZ[g];
    G.P = &T.box[T.gbox[g]];
    // |x_i - c| <= h and |x_j - c| < h + r_cut per axis, so x_j - x_i computed
    // from group-relative offsets is already the minimum image when
    // 2h + r_cut < 1/2; otherwise (tiny boxes) pair offsets are taken from the
    // integer images directly.
    const double hm = fmax(T.ghx[g], fmax(T.ghy[g], T.ghz[g]));
    G.wrap = 2.0 * hm + G.P->rcut >= 0.5 - 1e-9;
    return G;
}

// The number of work items: with an LPT order, every group's first chunk and
// the further chunks of larger groups (k_lpt_keys); without one, the groups.
__device__ __forceinline__ int64_t work_count(const TreeDev &T, const int32_t *order)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    if (!order) return G;
    const int64_t x = *T.n_xitems;
    return G + (x < T.cap_xitems ? x : T.cap_xitems);
}

// Work item `item`: with an LPT order the group's particles narrowed to the
// item's chunk of at most kWorkChunk (order values below cap_groups are the
// groups' first chunks, the others index the table of further chunks);
// without one, group `item` whole.  (One inlined load_group on both paths:
// an early return with a second copy made the packed forward kernel's
// register allocation and schedule worse, 1.7 % on the clustered 2M box.)
__device__ __forceinline__ Group load_work(const TreeDev &T, const int32_t *order, int64_t item)
{
    int64_t g = item;
    int i0 = 0;
    if (order) {
        const int64_t v = order[item];
        g = v;
        if (v >= T.cap_groups) {
            const int2 x = T.xitem[v - T.cap_groups];
            g = x.x;
            i0 = x.y * kWorkChunk;
        }
    }
    Group G = load_group(T, g);
    G.first += i0;
    G.ni = order ? min(kWorkChunk, G.ni - i0) : G.ni;
    return G;
}

// Shared-memory j tile: group-relative scaled offsets, or for groups that
// span half the box the raw 64-bit images (their pair differences are taken
// in integers, which is the exact minimum image).
template <class R>
struct JTile {
    union {
        struct { R x[kTile], y[kTile], z[kTile]; } f;
        struct { uint64_t x[kTile], y[kTile], z[kTile]; } u;
    };
    R m[kTile];
};

template <class R>
__device__ __forceinline__ void stage_entry(const TreeDev &T, const Group &G, int32_t e, R sc,
                                            JTile<R> &J, int q)
{
    uint64_t ex, ey, ez;
    double mj;
    if (e >= 0) {
        ex = T.X[e]; ey = T.Y[e]; ez = T.Z[e]; mj = T.m[e];
    } else {
        const int32_t nd = -e - 1;
        ex = T.cX[nd]; ey = T.cY[nd]; ez = T.cZ[nd]; mj = T.M[nd];
    }
    if (G.wrap) {
        J.u.x[q] = ex; J.u.y[q] = ey; J.u.z[q] = ez;
    } else {
        J.f.x[q] = Arith<R>::from_fixed(ex, G.X, sc);
        J.f.y[q] = Arith<R>::from_fixed(ey, G.Y, sc);
        J.f.z[q] = Arith<R>::from_fixed(ez, G.Z, sc);
    }
    J.m[q] = (R)mj;
}

// The i particle: its scaled group-relative offset and its raw images.
template <class R>
struct IPart {
    R x, y, z;
    uint64_t X, Y, Z;
};

template <class R, bool WRAP>
__device__ __forceinline__ void pair_offset(const JTile<R> &J, int j, const IPart<R> &I, R sc, R &dx,
                                            R &dy, R &dz)
{
    if (WRAP) {
        dx = Arith<R>::from_fixed(J.u.x[j], I.X, sc);
        dy = Arith<R>::from_fixed(J.u.y[j], I.Y, sc);
        dz = Arith<R>::from_fixed(J.u.z[j], I.Z, sc);
    } else {
        dx = J.f.x[j] - I.x;
        dy = J.f.y[j] - I.y;
        dz = J.f.z[j] - I.z;
    }
}

// Two pairs per step, packed.  Eq. 3 as g = u^5 h(xi) + v^6 c(xi) with
// u = max(0, 2 - xi), v = max(0, 1 - xi), h = (7 xi^3 + 22 xi^2 + 10 xi + 4)/140
// and c = (7 xi^2 + 18 xi + 3)/35: on [1,2] the first term alone is Eq. 3's
// factored form, on [0,1] the second adds Eq. 3's difference between its two
// branches, (1 - xi)^6 c(xi).  Both terms are non-negative (no cancellation in
// FP32) and u = 0 makes g vanish exactly at and beyond the cutoff.
// Two pairs per step, packed, for NI particles per thread: each staged entry
// pair (A = {x0, x1, y0, y1}, B = {z0, z1, m0, m1}) is loaded once and used
// for all NI particles.  Eq. 3 as g = u^5 h + v^6 c (exact 0 beyond the cutoff).
template <int NI, bool SOFT, bool RF>
__device__ __forceinline__ void force_tile_packed(const float4 *SA, const float4 *SB, int st, int npairs, int ns,
                                                  const float *xi, const float *yi, const float *zi, float eps2,
                                                  float *axs, float *ays, float *azs)
{
    f2 X[NI], Y[NI], Z[NI], ax[NI], ay[NI], az[NI];
#pragma unroll
    for (int k = 0; k < NI; k++) {
        X[k] = f2pack(xi[k], xi[k]); Y[k] = f2pack(yi[k], yi[k]); Z[k] = f2pack(zi[k], zi[k]);
        ax[k] = ay[k] = az[k] = f2pack(0.f, 0.f);
    }
    const f2 E2 = f2pack(eps2, eps2), TWO = f2pack(2.f, 2.f), ONE = f2pack(1.f, 1.f);
    const f2 H3 = f2pack(7.f / 140.f, 7.f / 140.f), H2 = f2pack(22.f / 140.f, 22.f / 140.f);
    const f2 H1 = f2pack(10.f / 140.f, 10.f / 140.f), H0 = f2pack(4.f / 140.f, 4.f / 140.f);
    const f2 C2 = f2pack(7.f / 35.f, 7.f / 35.f), C1 = f2pack(18.f / 35.f, 18.f / 35.f);
    const f2 C0 = f2pack(3.f / 35.f, 3.f / 35.f);
#pragma unroll 2
    for (int p = st; p < npairs; p += ns) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&SA[p]);
        const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&SB[p]);
#pragma unroll
        for (int k = 0; k < NI; k++) {
            const f2 dx = f2sub(a.x, X[k]), dy = f2sub(a.y, Y[k]), dz = f2sub(b.x, Z[k]);
            // the softened form needs only s^2 (eps^2 folded into the chain);
            // the self term vanishes through d = 0 in either form
            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, SOFT ? f2fma(dx, dx, E2) : f2mul(dx, dx)));
            const f2 s2 = SOFT ? r2 : f2add(r2, E2);
            float s2a, s2b;
            f2unpack(s2, s2a, s2b);
            const f2 ri = RF ? rsqrt_refined(s2) : f2pack(rsqrt_approx(s2a), rsqrt_approx(s2b));
            f2 x;                                   // the cutoff argument xi
            if (SOFT) {
                x = f2pack(sqrt_approx(s2a), sqrt_approx(s2b));
            } else {
                float r2a, r2b;
                f2unpack(r2, r2a, r2b);
                x = f2pack(sqrt_approx(r2a), sqrt_approx(r2b));
            }
            const f2 u = f2relu(f2sub(TWO, x));
            const f2 v = f2relu(f2sub(ONE, x));
            f2 h = f2fma(H3, x, H2);
            h = f2fma(h, x, H1);
            h = f2fma(h, x, H0);
            f2 c = f2fma(C2, x, C1);
            c = f2fma(c, x, C0);
            const f2 u2 = f2mul(u, u), v2 = f2mul(v, v);
            const f2 u5 = f2mul(f2mul(u2, u2), u), v6 = f2mul(f2mul(v2, v2), v2);
            const f2 g = f2fma(v6, c, f2mul(u5, h));
            const f2 ri3 = f2mul(f2mul(ri, ri), ri);
            const f2 f = f2mul(f2mul(b.y, g), ri3);
            ax[k] = f2fma(f, dx, ax[k]);
            ay[k] = f2fma(f, dy, ay[k]);
            az[k] = f2fma(f, dz, az[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < NI; k++) {
        float l, h;
        f2unpack(ax[k], l, h); axs[k] += l + h;
        f2unpack(ay[k], l, h); ays[k] += l + h;
        f2unpack(az[k], l, h); azs[k] += l + h;
    }
}

// g and g'/xi for two pairs at once, in the cancellation-free forms
// g = u^5 h + v^6 c and g'/xi = u^4 q' - (8/5) v^5 (xi + 2), with u = max(0,
// 2 - xi), v = max(0, 1 - xi), h = (7 xi^3 + 22 xi^2 + 10 xi + 4)/140,
// c = (7 xi^2 + 18 xi + 3)/35, q' = -(2 xi^2 + 4 xi - 1)/5.
__device__ __forceinline__ void g_gpx_packed(f2 x, f2 &g, f2 &gp)
{
    const f2 u = f2relu(f2sub(f2pack(2.f, 2.f), x));
    const f2 v = f2relu(f2sub(f2pack(1.f, 1.f), x));
    f2 h = f2fma(f2pack(7.f / 140.f, 7.f / 140.f), x, f2pack(22.f / 140.f, 22.f / 140.f));
    h = f2fma(h, x, f2pack(10.f / 140.f, 10.f / 140.f));
    h = f2fma(h, x, f2pack(4.f / 140.f, 4.f / 140.f));
    f2 c = f2fma(f2pack(7.f / 35.f, 7.f / 35.f), x, f2pack(18.f / 35.f, 18.f / 35.f));
    c = f2fma(c, x, f2pack(3.f / 35.f, 3.f / 35.f));
    f2 q = f2fma(f2pack(-2.f / 5.f, -2.f / 5.f), x, f2pack(-4.f / 5.f, -4.f / 5.f));
    q = f2fma(q, x, f2pack(1.f / 5.f, 1.f / 5.f));
    const f2 u2 = f2mul(u, u), u4 = f2mul(u2, u2), v2 = f2mul(v, v), v4 = f2mul(v2, v2);
    const f2 v5 = f2mul(v4, v);
    g = f2fma(f2mul(v4, v2), c, f2mul(f2mul(u4, u), h));
    const f2 xp = f2fma(x, f2pack(-8.f / 5.f, -8.f / 5.f), f2pack(-16.f / 5.f, -16.f / 5.f));
    gp = f2fma(v5, xp, f2mul(u4, q));
}

// hi + lo += x with the rounding error of the addition kept in lo (Knuth's
// TwoSum), so a long running sum in FP32 stays as accurate as one in FP64.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

template <class R>
__device__ __forceinline__ R scale_of(const BoxPrm &P);
template <> __device__ __forceinline__ float scale_of<float>(const BoxPrm &P) { return P.scale; }
template <> __device__ __forceinline__ double scale_of<double>(const BoxPrm &P)
{
    return P.scale_d * (2.0 / P.rcut);
}
template <class R>
__device__ __forceinline__ R eps2_of(const BoxPrm &P);
template <> __device__ __forceinline__ float eps2_of<float>(const BoxPrm &P) { return P.eps2s; }
template <> __device__ __forceinline__ double eps2_of<double>(const BoxPrm &P)
{
    const double k = 2.0 / P.rcut;
    return (k * P.eps) * (k * P.eps);
}

// Next work item: a persistent queue (atomic counter over an LPT order) or a
// plain grid-stride over groups.
template <bool QUEUE>
__device__ __forceinline__ int64_t next_item(int32_t *queue, int64_t cur, int *s_item)
{
    if (!QUEUE) return cur < 0 ? (int64_t)blockIdx.x : cur + gridDim.x;
    if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t it = *s_item;
    __syncthreads();
    return it;
}

template <class R, bool WRAP, bool SOFT>
__device__ __forceinline__ void force_tile(const JTile<R> &J, int st, int nt, int ns, const IPart<R> &I,
                                           R eps2, R sc, R &ax, R &ay, R &az)
{
    for (int j = st; j < nt; j += ns) {
        R dx, dy, dz;
        pair_offset<R, WRAP>(J, j, I, sc, dx, dy, dz);
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R s2 = r2 + eps2;
        const R ri = Arith<R>::rsqrt(s2);
        const R c2 = SOFT ? s2 : r2;            // xi^2: the plain or the softened |d'|^2
        const R x = SOFT ? Arith<R>::soft_xi(s2, ri) : Arith<R>::sqrt(r2);
        const R g = g_p3m<R>(x, c2);
        R f = J.m[j] * g * (ri * ri * ri);
        f = (c2 < R(4) && r2 > R(0)) ? f : R(0);
        ax += f * dx;
        ay += f * dy;
        az += f * dz;
    }
}

// ---------------------------------------------------------------------------
// Forward: a_i = G k^2 sum_j m_j d' g(|d'|) / (|d'|^2 + (k eps)^2)^{3/2}.
// ---------------------------------------------------------------------------
template <class R, bool QUEUE, bool SOFT>
__global__ void __launch_bounds__(kThreads) k_pair(TreeDev T, R *acc, int32_t *queue,
                                                   const int32_t *order)
{
    __shared__ JTile<R> J;
    __shared__ double red[3][kThreads];
    __shared__ int s_item;
    if (sizeof(R) == 4 && *T.n_general == 0) return;     // every group went to the packed kernel
    const int64_t W_n = work_count(T, order);
    const bool bad = *T.status == TP_ERR_LIST_OVERFLOW;
    for (int64_t item = next_item<QUEUE>(queue, -1, &s_item); item < W_n;
         item = next_item<QUEUE>(queue, item, &s_item)) {
        const Group G = load_work(T, order, item);
        const R sc = scale_of<R>(*G.P), eps2 = eps2_of<R>(*G.P);
        if (sizeof(R) == 4 && !G.wrap && eps2 > R(0)) continue;   // k_pair_packed takes these
        for (int i0 = 0; i0 < G.ni; i0 += kThreads) {
            const int nic = min(kThreads, G.ni - i0);
            const int ns = kThreads / nic;
            const int slot = threadIdx.x;
            const bool active = slot < nic * ns;
            const int il = active ? slot % nic : 0, st = active ? slot / nic : 0;
            const int32_t p = G.first + i0 + il;
            IPart<R> I;
            I.X = T.X[p]; I.Y = T.Y[p]; I.Z = T.Z[p];
            I.x = Arith<R>::from_fixed(I.X, G.X, sc);
            I.y = Arith<R>::from_fixed(I.Y, G.Y, sc);
            I.z = Arith<R>::from_fixed(I.Z, G.Z, sc);
            // Two-level accumulation: each tile's terms (at most kTile / ns per
            // thread) are summed in the working precision, tile sums in FP64.  A
            // list of thousands of nearly cancelling terms summed wholly in FP32
            // loses ~1e-5 relative; tile-sized partial sums keep it below 1e-6.
            double sax = 0.0, say = 0.0, saz = 0.0;
            const int ne = bad ? 0 : G.ne;
            for (int t0 = 0; t0 < ne; t0 += kTile) {
                const int nt = min(kTile, ne - t0);
                __syncthreads();
                for (int q = threadIdx.x; q < nt; q += kThreads)
                    stage_entry<R>(T, G, T.ent[G.e0 + t0 + q], sc, J, q);
                __syncthreads();
                if (active) {
                    R ax = 0, ay = 0, az = 0;
                    if (G.wrap) {
                        force_tile<R, true, SOFT>(J, st, nt, ns, I, eps2, sc, ax, ay, az);
                    } else {
                        force_tile<R, false, SOFT>(J, st, nt, ns, I, eps2, sc, ax, ay, az);
                    }
                    sax += (double)ax; say += (double)ay; saz += (double)az;
                }
            }
            red[0][slot] = sax; red[1][slot] = say; red[2][slot] = saz;
            __syncthreads();
            if (slot < nic) {
                double sxx = 0, syy = 0, szz = 0;
                for (int s = 0; s < ns; s++) {
                    sxx += red[0][s * nic + slot];
                    syy += red[1][s * nic + slot];
                    szz += red[2][s * nic + slot];
                }
                const int64_t o = T.perm[G.first + i0 + slot];
                acc[3 * o] = (R)(sxx * G.P->gk2);
                acc[3 * o + 1] = (R)(syy * G.P->gk2);
                acc[3 * o + 2] = (R)(szz * G.P->gk2);
            }
            __syncthreads();
        }
    }
}

// The FP32 forward kernel for ordinary groups with eps > 0: packed pair math
// fed by the entry records.  Each of the 128 threads holds NI particles of
// the work item (a group, or a chunk of at most kWorkChunk particles of a
// larger one) and takes a slice of the entry pairs of every tile (256
// entries): the item's particle columns (NI particles each) and the slices
// make a grid of columns x floor(128 / columns) threads, and the threads left
// over idle.
// Tiles are double buffered in shared memory:
// while tile t is computed from one buffer, each thread stores its entry pair
// of tile t+1 (loaded one tile earlier into registers) into the other buffer
// and loads its pair of tile t+2, so one barrier per tile suffices.  A tile
// holds 2 ns floor(128 / ns) entries (at most 256), so that each of the ns
// slices takes the same number of pairs from it.  The FP32
// partials of TS consecutive tiles enter an FP64 sum per particle: on GB300 a
// warp's FP64 add occupies its scheduler's FP64 unit for about 77 cycles, so
// adding every tile (TS = 1) stalls each warp for several hundred cycles per
// tile; TS = 8 (FP32 runs of at most 8 x 256 / slices entries per thread)
// measured 2 % faster on the clustered 2M box with the FP32 error unchanged
// (rms 4.1e-7 against the FP64 path on the same lists).
template <int NI, int TS, bool SOFT, bool RF>
__global__ void __launch_bounds__(kThreads) k_pair_packed(TreeDev T, float *acc, int32_t *queue,
                                                          const int32_t *order)
{
    constexpr int NT = kThreads;
    __shared__ float4 SA[2][NT], SB[2][NT];
    __shared__ double red[3 * NI][NT];
    __shared__ int s_item;
    const int64_t W_n = work_count(T, order);
    const bool bad = *T.status == TP_ERR_LIST_OVERFLOW;
    const float4 pad = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);
    for (int64_t item = next_item<true>(queue, -1, &s_item); item < W_n;
         item = next_item<true>(queue, item, &s_item)) {
        const Group G = load_work(T, order, item);
        const float sc = G.P->scale, eps2 = G.P->eps2s;
        if (G.wrap || !(eps2 > 0.f)) continue;              // the general kernel takes these
        const int ne = bad ? 0 : G.ne;
        for (int i0 = 0; i0 < G.ni; i0 += NI * NT) {
            // particle k*nip + il of this chunk goes to the threads il, il + nip, ... (slices)
            const int nic = min(NI * NT, G.ni - i0);
            const int nip = (nic + NI - 1) / NI;
            const int ns = NT / nip;
            const int slot = threadIdx.x;
            const bool active = slot < nip * ns;
            const int il = active ? slot % nip : 0, st = active ? slot / nip : 0;
            // entries per tile: a multiple of 2 ns, so that every slice takes
            // the same number of pairs of each full tile (the barrier after a
            // tile waits for the longest slice)
            const int kT = 2 * ns * (NT / ns);
            float xi[NI], yi[NI], zi[NI];
#pragma unroll
            for (int k = 0; k < NI; k++) {
                const int i = k * nip + il;
                if (i < nic) {
                    const int32_t p = G.first + i0 + i;
                    xi[k] = Arith<float>::from_fixed(T.X[p], G.X, sc);
                    yi[k] = Arith<float>::from_fixed(T.Y[p], G.Y, sc);
                    zi[k] = Arith<float>::from_fixed(T.Z[p], G.Z, sc);
                } else {                                   // a pad particle far from everything
                    xi[k] = yi[k] = zi[k] = -1.0e4f;
                }
            }
            double sax[NI], say[NI], saz[NI];
            float ax[NI], ay[NI], az[NI];
#pragma unroll
            for (int k = 0; k < NI; k++) {
                sax[k] = say[k] = saz[k] = 0.0;
                ax[k] = ay[k] = az[k] = 0.f;
            }
            float4 n0 = pad, n1 = pad;
            auto fetch = [&](int t1) {
                const int nt1 = min(kT, ne - t1), q = 2 * (int)threadIdx.x;
                n0 = q < nt1 ? T.rec[G.e0 + t1 + q] : pad;
                n1 = q + 1 < nt1 ? T.rec[G.e0 + t1 + q + 1] : pad;
            };
            // this thread's entry pair of a tile, staged as {x0, x1, y0, y1}, {z0, z1, m0, m1}
            auto stage = [&](int bb) {
                SA[bb][threadIdx.x] = make_float4(n0.x, n1.x, n0.y, n1.y);
                SB[bb][threadIdx.x] = make_float4(n0.z, n1.z, n0.w, n1.w);
            };
            __syncthreads();
            if (ne > 0) {
                fetch(0);
                stage(0);
                if (kT < ne) fetch(kT);
            }
            __syncthreads();
            int tc = 0;                                     // tiles in the current FP32 partial
            for (int t0 = 0, b = 0; t0 < ne; t0 += kT, b ^= 1) {
                const int nt = min(kT, ne - t0);
                if (active) {
                    force_tile_packed<NI, SOFT, RF>(SA[b], SB[b], st, (nt + 1) >> 1, ns, xi, yi, zi, eps2, ax, ay, az);
                    if (++tc == TS || t0 + kT >= ne) {
#pragma unroll
                        for (int k = 0; k < NI; k++) {
                            sax[k] += ax[k]; say[k] += ay[k]; saz[k] += az[k];
                            ax[k] = ay[k] = az[k] = 0.f;
                        }
                        tc = 0;
                    }
                }
                if (t0 + kT < ne) {
                    stage(b ^ 1);
                    if (t0 + 2 * kT < ne) fetch(t0 + 2 * kT);
                }
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < NI; k++) {
                red[3 * k][slot] = sax[k]; red[3 * k + 1][slot] = say[k]; red[3 * k + 2][slot] = saz[k];
            }
            __syncthreads();
            for (int i = slot; i < nic; i += NT) {
                const int k = i / nip, l = i % nip;
                double sxx = 0, syy = 0, szz = 0;
                for (int s2 = 0; s2 < ns; s2++) {
                    sxx += red[3 * k][s2 * nip + l];
                    syy += red[3 * k + 1][s2 * nip + l];
                    szz += red[3 * k + 2][s2 * nip + l];
                }
                const int64_t o = T.perm[G.first + i0 + i];
                acc[3 * o] = (float)(sxx * G.P->gk2);
                acc[3 * o + 1] = (float)(syy * G.P->gk2);
                acc[3 * o + 2] = (float)(szz * G.P->gk2);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint.  With f(d') = d' phi, phi = g(xi)/s'^3, s'^2 = xi^2 + (k eps)^2:
//   J' = phi I + psi d' d'^T,  psi = (g'/xi)/s'^3 - 3 g/s'^5,
//   v  = m_j J' w_i = alpha w_i + beta d',  alpha = m_j phi, beta = m_j psi (d'.w_i)
// and dL/dx_i -= G k^3 v, dL/dx_j += G k^3 v (a node passes its share to its
// centre-of-mass cotangent); the kernels add -v and +v, and the common factor
// G k^3 of a box is applied per particle at the end (k_unsort_grad).
// Threads hold list entries (j) and loop over the group's particles (i) held
// in shared memory, so the j side sums in registers; the i side (A_i = sum
// alpha, B_i = sum beta d') is reduce-scattered across each warp and summed
// over the tiles in compensated FP32 (the kernels below).
// ---------------------------------------------------------------------------

// g and g'/xi in the cancellation-free form (u = max(0, 2 - xi),
// v = max(0, 1 - xi)): g = u^5 (7 xi^3 + 22 xi^2 + 10 xi + 4)/140 + v^6 (7 xi^2
// + 18 xi + 3)/35 and g'/xi = -u^4 (2 xi^2 + 4 xi - 1)/5 - (8/5) v^5 (xi + 2).
// The second can lose ~2e-7 absolute near xi = 0, where it enters J only
// multiplied by xi^2.
template <class R>
__device__ __forceinline__ void g_gpx(R x, R &g, R &gp)
{
    const R u = fmax(R(2) - x, R(0)), v = fmax(R(1) - x, R(0));
    R h = R(7.0 / 140.0) * x + R(22.0 / 140.0);
    h = h * x + R(10.0 / 140.0);
    h = h * x + R(4.0 / 140.0);
    R c = R(7.0 / 35.0) * x + R(18.0 / 35.0);
    c = c * x + R(3.0 / 35.0);
    const R u2 = u * u, u4 = u2 * u2, v2 = v * v, v4 = v2 * v2;
    g = v4 * v2 * c + u4 * u * h;
    R q = R(2.0 / 5.0) * x + R(4.0 / 5.0);
    q = q * x + R(-1.0 / 5.0);
    gp = -(u4 * q) - R(8.0 / 5.0) * (v4 * v) * (x + R(2));
}

template <class R, bool SOFT>
__global__ void __launch_bounds__(kThreads) k_vjp(TreeDev T, const R *cot, double *gs, double *ncot,
                                                  int32_t *queue, const int32_t *order)
{
    __shared__ R ix[kThreads], iy[kThreads], iz[kThreads], iwx[kThreads], iwy[kThreads], iwz[kThreads];
    __shared__ uint64_t iX[kThreads], iY[kThreads], iZ[kThreads];
    __shared__ R part[kThreads / 32][4][kThreads];   // per-warp i-side sums of one tile
    __shared__ int s_item;
    if (sizeof(R) == 4 && *T.n_general == 0) return;     // every group went to the packed kernel
    const int64_t W_n = work_count(T, order);
    const bool bad = *T.status == TP_ERR_LIST_OVERFLOW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t item = next_item<true>(queue, -1, &s_item); item < W_n;
         item = next_item<true>(queue, item, &s_item)) {
        const Group G = load_work(T, order, item);
        const R sc = scale_of<R>(*G.P), eps2 = eps2_of<R>(*G.P);
        if (sizeof(R) == 4 && !G.wrap && eps2 > R(0)) continue;   // k_vjp_fused takes these
        const int ne = bad ? 0 : G.ne;
        for (int i0 = 0; i0 < G.ni; i0 += kThreads) {
            const int nic = min(kThreads, G.ni - i0);
            if (threadIdx.x < nic) {
                const int32_t p = G.first + i0 + threadIdx.x;
                const uint64_t X = T.X[p], Y = T.Y[p], Z = T.Z[p];
                iX[threadIdx.x] = X; iY[threadIdx.x] = Y; iZ[threadIdx.x] = Z;
                ix[threadIdx.x] = Arith<R>::from_fixed(X, G.X, sc);
                iy[threadIdx.x] = Arith<R>::from_fixed(Y, G.Y, sc);
                iz[threadIdx.x] = Arith<R>::from_fixed(Z, G.Z, sc);
                const int64_t o = T.perm[p];
                iwx[threadIdx.x] = cot[3 * o]; iwy[threadIdx.x] = cot[3 * o + 1]; iwz[threadIdx.x] = cot[3 * o + 2];
            }
            // thread t < nic owns particle i0 + t's i-side sums (FP64 across tiles)
            double sA = 0.0, sBx = 0.0, sBy = 0.0, sBz = 0.0;
            __syncthreads();
            for (int t0 = 0; t0 < ne; t0 += kThreads) {
                const int q = t0 + threadIdx.x;
                const bool valid = q < ne;
                int32_t e = 0;
                uint64_t ex = 0, ey = 0, ez = 0;
                R mj = 0;
                if (valid) {
                    e = T.ent[G.e0 + q];
                    if (e >= 0) {
                        ex = T.X[e]; ey = T.Y[e]; ez = T.Z[e]; mj = (R)T.m[e];
                    } else {
                        const int32_t nd = -e - 1;
                        ex = T.cX[nd]; ey = T.cY[nd]; ez = T.cZ[nd]; mj = (R)T.M[nd];
                    }
                }
                const R xj = Arith<R>::from_fixed(ex, G.X, sc), yj = Arith<R>::from_fixed(ey, G.Y, sc),
                        zj = Arith<R>::from_fixed(ez, G.Z, sc);
                R vx = 0, vy = 0, vz = 0;
                for (int k = 0; k < nic; k++) {
                    R dx, dy, dz;
                    if (G.wrap) {
                        dx = Arith<R>::from_fixed(ex, iX[k], sc);
                        dy = Arith<R>::from_fixed(ey, iY[k], sc);
                        dz = Arith<R>::from_fixed(ez, iZ[k], sc);
                    } else {
                        dx = xj - ix[k]; dy = yj - iy[k]; dz = zj - iz[k];
                    }
                    const R wx = iwx[k], wy = iwy[k], wz = iwz[k];
                    const R r2 = dx * dx + dy * dy + dz * dz;
                    const R s2 = r2 + eps2;
                    const R ri = Arith<R>::rsqrt(s2);
                    const R x = SOFT ? Arith<R>::soft_xi(s2, ri) : Arith<R>::sqrt(r2);
                    R gv, gp;
                    g_gpx<R>(x, gv, gp);
                    const R ri2 = ri * ri, ri3 = ri2 * ri;
                    const R phi = gv * ri3;
                    const R psi = gp * ri3 - R(3) * phi * ri2;
                    const bool in = valid && r2 > R(0);
                    const R alpha = in ? mj * phi : R(0);
                    const R beta = in ? mj * psi * (dx * wx + dy * wy + dz * wz) : R(0);
                    vx += alpha * wx + beta * dx;
                    vy += alpha * wy + beta * dy;
                    vz += alpha * wz + beta * dz;
                    R a = alpha, bx = beta * dx, by = beta * dy, bz = beta * dz;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, off);
                        bx += __shfl_xor_sync(0xffffffffu, bx, off);
                        by += __shfl_xor_sync(0xffffffffu, by, off);
                        bz += __shfl_xor_sync(0xffffffffu, bz, off);
                    }
                    if (lane == 0) {
                        part[warp][0][k] = a; part[warp][1][k] = bx;
                        part[warp][2][k] = by; part[warp][3][k] = bz;
                    }
                }
                if (valid) {
                    double *dst = e >= 0 ? gs + 3 * (int64_t)e : ncot + 3 * (int64_t)(-e - 1);
                    atomicAdd(dst, (double)vx);
                    atomicAdd(dst + 1, (double)vy);
                    atomicAdd(dst + 2, (double)vz);
                }
                __syncthreads();
                if (threadIdx.x < nic) {
                    const int nw = min(kThreads, ne - t0 + 31) >> 5;   // warps that held entries
                    for (int w = 0; w < nw; w++) {
                        sA += (double)part[w][0][threadIdx.x]; sBx += (double)part[w][1][threadIdx.x];
                        sBy += (double)part[w][2][threadIdx.x]; sBz += (double)part[w][3][threadIdx.x];
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x < nic) {
                const int32_t p = G.first + i0 + threadIdx.x;
                atomicAdd(gs + 3 * (int64_t)p, -(sA * (double)iwx[threadIdx.x] + sBx));
                atomicAdd(gs + 3 * (int64_t)p + 1, -(sA * (double)iwy[threadIdx.x] + sBy));
                atomicAdd(gs + 3 * (int64_t)p + 2, -(sA * (double)iwz[threadIdx.x] + sBz));
            }
            __syncthreads();
        }
    }
}

// Adjoint for ordinary groups with eps > 0 (FP32, packed): threads hold list
// entries and loop over the group's particles two at a time, staged as
// A = {x0, x1, y0, y1}, B = {z0, z1, wx0, wx1}, C = {wy0, wy1, wz0, wz1}.  Each
// pair's alpha = m phi and beta = m psi (d.w_i) are computed once: the entry
// sums its side, v = sum_i (alpha w_i + beta d), in registers.  The particle
// side, A_i = sum alpha and B_i = sum beta d, is summed over the warp's 32
// entries for two particle pairs at once: their 16 values are reduce-scattered
// (four halving exchanges and one final one, 16 shuffles in all) so that each
// lane pair ends with one total, written to the warp's row; the thread that
// owns the particle adds the rows and keeps a compensated FP32 sum across
// tiles.  Each thread holds E list entries (a tile is E x 128 entries) and
// adds their particle-side values before the reduce-scatter, so its cost is
// shared by E entries.
template <int E, bool FWD, bool SOFT, bool RF>
__global__ void __launch_bounds__(kThreads, E >= 4 ? 4 : (FWD ? 5 : 6)) k_vjp_fused(TreeDev T, const float *cot, double *gs, double *ncot,
                                                        int32_t *queue, const int32_t *order, float *acc)
{
    constexpr int kWarps = kThreads / 32;
    constexpr unsigned kFull = 0xffffffffu;
    // particle-side quantities: A = sum alpha, B = sum beta d (3), with FWD also
    // F = sum alpha d (3), the forward sum of Eq. 2 (alpha = m g / s^3)
    constexpr int NQ = FWD ? 7 : 4;
    constexpr int NV = FWD ? 32 : 16;      // values of two particle pairs (padded)
    __shared__ float4 IA[kThreads / 2], IB[kThreads / 2], IC[kThreads / 2];
    __shared__ float part[kWarps][NQ][kThreads];
    __shared__ int s_item;
    const int64_t W_n = work_count(T, order);
    const bool bad = *T.status == TP_ERR_LIST_OVERFLOW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // after the reduce-scatter below, lane holds the sum of value vidx:
    // value 8P + 2q + h (16 values) or 16P + 2q + h (32 values, FWD)
    const int vidx = FWD ? lane : (lane >> 1) & 15;
    const int vP = FWD ? vidx >> 4 : vidx >> 3, vq = FWD ? (vidx >> 1) & 7 : (vidx >> 1) & 3, vh = vidx & 1;
    for (int64_t item = next_item<true>(queue, -1, &s_item); item < W_n;
         item = next_item<true>(queue, item, &s_item)) {
        const Group G = load_work(T, order, item);
        const float sc = G.P->scale, eps2 = G.P->eps2s;
        if (G.wrap || !(eps2 > 0.f)) continue;              // the general kernel takes these
        const int ne = bad ? 0 : G.ne;
        for (int i0 = 0; i0 < G.ni; i0 += kThreads) {
            const int nic = min(kThreads, G.ni - i0);
            const int npr = (nic + 1) >> 1;                    // particle pairs holding particles
            const int npe = (npr + 1) & ~1;                    // particle pairs, rounded up to even
            __syncthreads();
            if (threadIdx.x < 2 * npe) {
                const int l = threadIdx.x & 1;
                float *A = reinterpret_cast<float *>(&IA[threadIdx.x >> 1]);
                float *B = reinterpret_cast<float *>(&IB[threadIdx.x >> 1]);
                float *Cc = reinterpret_cast<float *>(&IC[threadIdx.x >> 1]);
                if (threadIdx.x < nic) {
                    const int32_t p = G.first + i0 + threadIdx.x;
                    const int64_t o = T.perm[p];
                    A[l] = Arith<float>::from_fixed(T.X[p], G.X, sc);
                    A[2 + l] = Arith<float>::from_fixed(T.Y[p], G.Y, sc);
                    B[l] = Arith<float>::from_fixed(T.Z[p], G.Z, sc);
                    B[2 + l] = cot[3 * o]; Cc[l] = cot[3 * o + 1]; Cc[2 + l] = cot[3 * o + 2];
                } else {                                     // pad: far away, zero cotangent
                    A[l] = 1.0e4f; A[2 + l] = 1.0e4f; B[l] = 1.0e4f;
                    B[2 + l] = 0.f; Cc[l] = 0.f; Cc[2 + l] = 0.f;
                }
            }
            // particle-side sums across tiles, compensated FP32 (hi + lo)
            float sh[NQ], sl[NQ];
#pragma unroll
            for (int q = 0; q < NQ; q++) sh[q] = sl[q] = 0.f;
            __syncthreads();
            for (int t0 = 0; t0 < ne; t0 += E * kThreads) {
                int32_t e[E];
                f2 XJ[E], YJ[E], ZJ[E];
                float MJ[E];
                f2 vx[E], vy[E], vz[E];
#pragma unroll
                for (int u = 0; u < E; u++) {
                    const int q = t0 + u * kThreads + threadIdx.x;
                    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
                    e[u] = 0;
                    if (q < ne) {
                        e[u] = T.ent[G.e0 + q];
                        r = T.rec[G.e0 + q];
                    }
                    XJ[u] = f2pack(r.x, r.x); YJ[u] = f2pack(r.y, r.y); ZJ[u] = f2pack(r.z, r.z);
                    MJ[u] = r.w;                               // 0 for an empty slot
                    vx[u] = vy[u] = vz[u] = f2pack(0.f, 0.f);
                }
                const f2 E2 = f2pack(eps2, eps2), M3 = f2pack(-3.f, -3.f);
                const bool wfull = t0 + (E - 1) * kThreads + warp * 32 + 31 < ne;
                for (int pp = 0; pp < npe; pp += 2) {
                    float v[NV];
#pragma unroll
                    for (int P = 0; P < 2; P++) {
                        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(&IA[pp + P]);
                        const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&IB[pp + P]);
                        const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(&IC[pp + P]);
                        const f2 WX = b.y, WY = c.x, WZ = c.y;
                        f2 sa = f2pack(0.f, 0.f), sbx = sa, sby = sa, sbz = sa, sfx = sa, sfy = sa, sfz = sa;
                        // warp-uniform skips, whose terms would be exact zeros: the
                        // padding pair of an odd count of particle pairs, and the
                        // entry slots past the end of the list
                        const bool live = P == 0 || pp + 1 < npr;
                        auto term = [&](int u) {
                            const f2 dx = f2sub(XJ[u], a.x), dy = f2sub(YJ[u], a.y), dz = f2sub(ZJ[u], b.x);
                            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
                            const f2 s2 = f2add(r2, E2);
                            float r2a, r2b, s2a, s2b;
                            f2unpack(r2, r2a, r2b);
                            f2unpack(s2, s2a, s2b);
                            const f2 ri = RF ? rsqrt_refined(s2) : f2pack(rsqrt_approx(s2a), rsqrt_approx(s2b));
                            const f2 x = SOFT ? f2pack(sqrt_approx(s2a), sqrt_approx(s2b))   // xi
                                              : f2pack(sqrt_approx(r2a), sqrt_approx(r2b));
                            f2 gv, gp;
                            g_gpx_packed(x, gv, gp);
                            const f2 ri2 = f2mul(ri, ri);
                            // m_j / s'^3, zero for the particle itself (and coincident pairs)
                            const f2 mr3 = f2mul(f2pack(r2a > 0.f ? MJ[u] : 0.f, r2b > 0.f ? MJ[u] : 0.f),
                                                 f2mul(ri2, ri));
                            const f2 dw = f2fma(dz, WZ, f2fma(dy, WY, f2mul(dx, WX)));
                            const f2 alpha = f2mul(gv, mr3);                       // m phi
                            const f2 beta = f2mul(f2mul(f2fma(gv, f2mul(M3, ri2), gp), mr3), dw);   // m psi (d.w)
                            vx[u] = f2fma(beta, dx, f2fma(alpha, WX, vx[u]));
                            vy[u] = f2fma(beta, dy, f2fma(alpha, WY, vy[u]));
                            vz[u] = f2fma(beta, dz, f2fma(alpha, WZ, vz[u]));
                            sa = f2add(sa, alpha);
                            sbx = f2fma(beta, dx, sbx);
                            sby = f2fma(beta, dy, sby);
                            sbz = f2fma(beta, dz, sbz);
                            if (FWD) {
                                sfx = f2fma(alpha, dx, sfx);
                                sfy = f2fma(alpha, dy, sfy);
                                sfz = f2fma(alpha, dz, sfz);
                            }
                        };
                        // every slot of this warp holds an entry (all tiles but
                        // the last): no branch between the E independent terms
                        if (live && wfull) {
#pragma unroll
                            for (int u = 0; u < E; u++) term(u);
                        } else if (live) {
#pragma unroll
                            for (int u = 0; u < E; u++) {
                                if (t0 + u * kThreads + warp * 32 >= ne) break;
                                term(u);
                            }
                        }
                        constexpr int B0 = FWD ? 16 : 8;
                        f2unpack(sa, v[B0 * P + 0], v[B0 * P + 1]);
                        f2unpack(sbx, v[B0 * P + 2], v[B0 * P + 3]);
                        f2unpack(sby, v[B0 * P + 4], v[B0 * P + 5]);
                        f2unpack(sbz, v[B0 * P + 6], v[B0 * P + 7]);
                        if (FWD) {
                            f2unpack(sfx, v[B0 * P + 8], v[B0 * P + 9]);
                            f2unpack(sfy, v[B0 * P + 10], v[B0 * P + 11]);
                            f2unpack(sfz, v[B0 * P + 12], v[B0 * P + 13]);
                            v[B0 * P + 14] = 0.f;
                            v[B0 * P + 15] = 0.f;
                        }
                    }
                    // reduce-scatter over the warp's 32 lanes: each halving step
                    // keeps the half of the values selected by one lane bit
                    constexpr int kLevels = FWD ? 5 : 4;
#pragma unroll
                    for (int lvl = 0; lvl < kLevels; lvl++) {
                        const int off = 16 >> lvl, half = (NV / 2) >> lvl;
                        const bool upper = (lane & off) != 0;
#pragma unroll
                        for (int kk = 0; kk < half; kk++) {
                            const float send = upper ? v[kk] : v[kk + half];
                            const float keep = upper ? v[kk + half] : v[kk];
                            v[kk] = keep + __shfl_xor_sync(kFull, send, off);
                        }
                    }
                    if (FWD) {
                        if (vq < NQ) part[warp][vq][2 * (pp + vP) + vh] = v[0];
                    } else {
                        v[0] += __shfl_xor_sync(kFull, v[0], 1);
                        if ((lane & 1) == 0) part[warp][vq][2 * (pp + vP) + vh] = v[0];
                    }
                }
#pragma unroll
                for (int u = 0; u < E; u++) {
                    if (t0 + u * kThreads + (int)threadIdx.x < ne) {
                        float l, h;
                        double *dst = e[u] >= 0 ? gs + 3 * (int64_t)e[u] : ncot + 3 * (int64_t)(-e[u] - 1);
                        f2unpack(vx[u], l, h); atomicAdd(dst, (double)(l + h));
                        f2unpack(vy[u], l, h); atomicAdd(dst + 1, (double)(l + h));
                        f2unpack(vz[u], l, h); atomicAdd(dst + 2, (double)(l + h));
                    }
                }
                __syncthreads();
                if (threadIdx.x < nic) {
                    const int nw = (min(kThreads, ne - t0) + 31) >> 5;   // warps that held entries
#pragma unroll
                    for (int k = 0; k < NQ; k++) {
                        float t = 0.f;
                        for (int w = 0; w < nw; w++) t += part[w][k][threadIdx.x];
                        two_sum_add(sh[k], sl[k], t);
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x < nic) {
                const int32_t p = G.first + i0 + threadIdx.x;
                const int64_t o = T.perm[p];
                const double sA = (double)sh[0] + (double)sl[0];
                atomicAdd(gs + 3 * (int64_t)p, -(sA * (double)cot[3 * o] + ((double)sh[1] + (double)sl[1])));
                atomicAdd(gs + 3 * (int64_t)p + 1, -(sA * (double)cot[3 * o + 1] + ((double)sh[2] + (double)sl[2])));
                atomicAdd(gs + 3 * (int64_t)p + 2, -(sA * (double)cot[3 * o + 2] + ((double)sh[3] + (double)sl[3])));
                if (FWD) {
                    const double gk2 = G.P->gk2;
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        acc[3 * o + c] = (float)(gk2 * ((double)sh[4 + c] + (double)sl[4 + c]));
                }
            }
        }
    }
}

// The same adjoint (with FWD, the forward sum too) with two list entries,
// not two particles, in each f32x2 operation.  Each thread holds EP pairs of
// entries (2 EP entries: a tile is 2 EP x 128), and the work item's particles
// are staged in shared memory with every value duplicated, {x, x, y, y},
// {z, z, wx, wx}, {wy, wy, wz, wz}, so that a particle enters both halves of
// a pair without a move.  The entry side v sums in registers per pair (its
// halves are two entries).  The particle side sums over the thread's pairs
// in packed form, then over the two halves, and the warp reduce-scatters 16
// values per step: two particles' 7 quantities (FWD) or four particles' 4.
// One reduce-scatter thus serves 2 EP entries of a thread instead of E, which
// halves its shuffles, selects and adds per interaction at EP = 4, in about
// the registers of k_vjp_fused<4>: a pair's offsets hold two entries rather
// than one entry twice.
template <int EP, bool FWD, bool SOFT, bool RF>
__global__ void __launch_bounds__(kThreads, 4) k_vjp_epack(TreeDev T, const float *cot, double *gs, double *ncot,
                                                           int32_t *queue, const int32_t *order, float *acc)
{
    constexpr int kWarps = kThreads / 32;
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int NQ = FWD ? 7 : 4;          // A, B (3), with FWD also F (3)
    constexpr int NP = FWD ? 2 : 4;          // particles per reduce-scatter
    constexpr int kSlot = FWD ? 8 : 4;       // values per particle in it (FWD: one padding)
    constexpr int kRow = 2 * kThreads;       // entries of one pair slot across the CTA
    __shared__ ulonglong2 IA[kThreads], IB[kThreads], IC[kThreads];
    __shared__ float part[kWarps][NQ][kThreads];
    __shared__ int s_item;
    const int64_t W_n = work_count(T, order);
    const bool bad = *T.status == TP_ERR_LIST_OVERFLOW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // after the reduce-scatter, lanes 2m and 2m+1 hold value m = kSlot P + q
    const int vidx = (lane >> 1) & 15;
    const int vP = vidx / kSlot, vq = vidx % kSlot;
    for (int64_t item = next_item<true>(queue, -1, &s_item); item < W_n;
         item = next_item<true>(queue, item, &s_item)) {
        const Group G = load_work(T, order, item);
        const float sc = G.P->scale, eps2 = G.P->eps2s;
        if (G.wrap || !(eps2 > 0.f)) continue;              // the general kernel takes these
        const int ne = bad ? 0 : G.ne;
        for (int i0 = 0; i0 < G.ni; i0 += kThreads) {
            const int nic = min(kThreads, G.ni - i0);
            const int npad = (nic + NP - 1) / NP * NP;      // particles rounded up to the step
            __syncthreads();
            if (threadIdx.x < npad) {
                float x = 1.0e4f, y = 1.0e4f, z = 1.0e4f, wx = 0.f, wy = 0.f, wz = 0.f;   // pad: far, no weight
                if (threadIdx.x < nic) {
                    const int32_t p = G.first + i0 + threadIdx.x;
                    const int64_t o = T.perm[p];
                    x = Arith<float>::from_fixed(T.X[p], G.X, sc);
                    y = Arith<float>::from_fixed(T.Y[p], G.Y, sc);
                    z = Arith<float>::from_fixed(T.Z[p], G.Z, sc);
                    wx = cot[3 * o]; wy = cot[3 * o + 1]; wz = cot[3 * o + 2];
                }
                IA[threadIdx.x] = make_ulonglong2(f2pack(x, x), f2pack(y, y));
                IB[threadIdx.x] = make_ulonglong2(f2pack(z, z), f2pack(wx, wx));
                IC[threadIdx.x] = make_ulonglong2(f2pack(wy, wy), f2pack(wz, wz));
            }
            float sh[NQ], sl[NQ];                           // compensated FP32 sums across tiles
#pragma unroll
            for (int q = 0; q < NQ; q++) sh[q] = sl[q] = 0.f;
            __syncthreads();
            for (int t0 = 0; t0 < ne; t0 += EP * kRow) {
                f2 XJ[EP], YJ[EP], ZJ[EP], MJ[EP], vx[EP], vy[EP], vz[EP];
#pragma unroll
                for (int u = 0; u < EP; u++) {
                    const int q = t0 + u * kRow + 2 * (int)threadIdx.x;
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 r0 = q < ne ? T.rec[G.e0 + q] : z4;
                    const float4 r1 = q + 1 < ne ? T.rec[G.e0 + q + 1] : z4;
                    XJ[u] = f2pack(r0.x, r1.x); YJ[u] = f2pack(r0.y, r1.y); ZJ[u] = f2pack(r0.z, r1.z);
                    MJ[u] = f2pack(r0.w, r1.w);                 // 0 for an empty slot
                    vx[u] = vy[u] = vz[u] = f2pack(0.f, 0.f);
                }
                const f2 E2 = f2pack(eps2, eps2), M3 = f2pack(-3.f, -3.f);
                const bool wfull = t0 + (EP - 1) * kRow + 64 * warp + 63 < ne;
                for (int k0 = 0; k0 < npad; k0 += NP) {
                    float v[16];
#pragma unroll
                    for (int P = 0; P < NP; P++) {
                        const ulonglong2 a = IA[k0 + P], b = IB[k0 + P], c = IC[k0 + P];
                        const f2 X = a.x, Y = a.y, Z = b.x, WX = b.y, WY = c.x, WZ = c.y;
                        f2 sa = f2pack(0.f, 0.f), sbx = sa, sby = sa, sbz = sa, sfx = sa, sfy = sa, sfz = sa;
                        auto term = [&](int u) {
                            const f2 dx = f2sub(XJ[u], X), dy = f2sub(YJ[u], Y), dz = f2sub(ZJ[u], Z);
                            const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
                            const f2 s2 = f2add(r2, E2);
                            float r2a, r2b, s2a, s2b, ma, mb;
                            f2unpack(r2, r2a, r2b);
                            f2unpack(s2, s2a, s2b);
                            f2unpack(MJ[u], ma, mb);
                            const f2 ri = RF ? rsqrt_refined(s2) : f2pack(rsqrt_approx(s2a), rsqrt_approx(s2b));
                            const f2 x = SOFT ? f2pack(sqrt_approx(s2a), sqrt_approx(s2b))   // xi
                                              : f2pack(sqrt_approx(r2a), sqrt_approx(r2b));
                            f2 gv, gp;
                            g_gpx_packed(x, gv, gp);
                            const f2 ri2 = f2mul(ri, ri);
                            // m_j / s'^3, zero for the particle itself (and coincident pairs)
                            const f2 mr3 = f2mul(f2pack(r2a > 0.f ? ma : 0.f, r2b > 0.f ? mb : 0.f), f2mul(ri2, ri));
                            const f2 dw = f2fma(dz, WZ, f2fma(dy, WY, f2mul(dx, WX)));
                            const f2 alpha = f2mul(gv, mr3);                       // m phi
                            const f2 beta = f2mul(f2mul(f2fma(gv, f2mul(M3, ri2), gp), mr3), dw);   // m psi (d.w)
                            vx[u] = f2fma(beta, dx, f2fma(alpha, WX, vx[u]));
                            vy[u] = f2fma(beta, dy, f2fma(alpha, WY, vy[u]));
                            vz[u] = f2fma(beta, dz, f2fma(alpha, WZ, vz[u]));
                            sa = f2add(sa, alpha);
                            sbx = f2fma(beta, dx, sbx);
                            sby = f2fma(beta, dy, sby);
                            sbz = f2fma(beta, dz, sbz);
                            if (FWD) {
                                sfx = f2fma(alpha, dx, sfx);
                                sfy = f2fma(alpha, dy, sfy);
                                sfz = f2fma(alpha, dz, sfz);
                            }
                        };
                        // warp-uniform skips of terms that would be exact zeros: padding
                        // particles, and pair slots of this warp past the list's end
                        if (k0 + P < nic) {
                            if (wfull) {
#pragma unroll
                                for (int u = 0; u < EP; u++) term(u);
                            } else {
#pragma unroll
                                for (int u = 0; u < EP; u++) {
                                    if (t0 + u * kRow + 64 * warp >= ne) break;
                                    term(u);
                                }
                            }
                        }
                        float l, h;
                        f2unpack(sa, l, h); v[kSlot * P + 0] = l + h;
                        f2unpack(sbx, l, h); v[kSlot * P + 1] = l + h;
                        f2unpack(sby, l, h); v[kSlot * P + 2] = l + h;
                        f2unpack(sbz, l, h); v[kSlot * P + 3] = l + h;
                        if (FWD) {
                            f2unpack(sfx, l, h); v[kSlot * P + 4] = l + h;
                            f2unpack(sfy, l, h); v[kSlot * P + 5] = l + h;
                            f2unpack(sfz, l, h); v[kSlot * P + 6] = l + h;
                            v[kSlot * P + 7] = 0.f;
                        }
                    }
                    // reduce-scatter of the 16 values over the warp's 32 lanes
#pragma unroll
                    for (int lvl = 0; lvl < 4; lvl++) {
                        const int off = 16 >> lvl, half = 8 >> lvl;
                        const bool upper = (lane & off) != 0;
#pragma unroll
                        for (int kk = 0; kk < half; kk++) {
                            const float send = upper ? v[kk] : v[kk + half];
                            const float keep = upper ? v[kk + half] : v[kk];
                            v[kk] = keep + __shfl_xor_sync(kFull, send, off);
                        }
                    }
                    v[0] += __shfl_xor_sync(kFull, v[0], 1);
                    if ((lane & 1) == 0 && vq < NQ) part[warp][vq][k0 + vP] = v[0];
                }
#pragma unroll
                for (int u = 0; u < EP; u++) {
                    const int q = t0 + u * kRow + 2 * (int)threadIdx.x;
                    float l, h;
                    if (q < ne) {
                        const int32_t e = T.ent[G.e0 + q];
                        double *dst = e >= 0 ? gs + 3 * (int64_t)e : ncot + 3 * (int64_t)(-e - 1);
                        f2unpack(vx[u], l, h); atomicAdd(dst, (double)l);
                        f2unpack(vy[u], l, h); atomicAdd(dst + 1, (double)l);
                        f2unpack(vz[u], l, h); atomicAdd(dst + 2, (double)l);
                    }
                    if (q + 1 < ne) {
                        const int32_t e = T.ent[G.e0 + q + 1];
                        double *dst = e >= 0 ? gs + 3 * (int64_t)e : ncot + 3 * (int64_t)(-e - 1);
                        f2unpack(vx[u], l, h); atomicAdd(dst, (double)h);
                        f2unpack(vy[u], l, h); atomicAdd(dst + 1, (double)h);
                        f2unpack(vz[u], l, h); atomicAdd(dst + 2, (double)h);
                    }
                }
                __syncthreads();
                if (threadIdx.x < nic) {
#pragma unroll
                    for (int k = 0; k < NQ; k++) {
                        float t = 0.f;
#pragma unroll
                        for (int w = 0; w < kWarps; w++) t += part[w][k][threadIdx.x];
                        two_sum_add(sh[k], sl[k], t);
                    }
                }
                __syncthreads();
            }
            if (threadIdx.x < nic) {
                const int32_t p = G.first + i0 + threadIdx.x;
                const int64_t o = T.perm[p];
                const double sA = (double)sh[0] + (double)sl[0];
                atomicAdd(gs + 3 * (int64_t)p, -(sA * (double)cot[3 * o] + ((double)sh[1] + (double)sl[1])));
                atomicAdd(gs + 3 * (int64_t)p + 1, -(sA * (double)cot[3 * o + 1] + ((double)sh[2] + (double)sl[2])));
                atomicAdd(gs + 3 * (int64_t)p + 2, -(sA * (double)cot[3 * o + 2] + ((double)sh[3] + (double)sl[3])));
                if (FWD) {
                    const double gk2 = G.P->gk2;
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        acc[3 * o + c] = (float)(gk2 * ((double)sh[4 + c] + (double)sl[4 + c]));
                }
            }
        }
    }
}

// Node cotangents reach member particles through the centre of mass: with
// q_a = c_a / M_a (taken as c_a times 1/M_a; 0 for an empty node) and
// P_a = P_parent(a) + q_a from the roots down, P at a leaf is the sum of q
// over its ancestors in root-to-leaf order, and grad_p += m_p P_leaf(p).
// k_node_quot turns every node's c into q in place; k_leaf_sum forms each
// leaf's P from its chain of parents (at most TP_NLEVELS nodes), stores it in
// the leaf's own slot (no other chain reads a leaf) and records the leaf of
// each of its particles; k_unsort_grad then adds m_p P per particle and
// writes the gradient in input order, with the box's factor G k^3, which the
// pair kernels leave out of their sums so that its FP64 multiply is taken
// once per particle here instead of once per entry and tile.
__global__ void k_node_quot(TreeDev T, double *ncot)
{
    const int64_t nn = *T.n_nodes < T.cap_nodes ? *T.n_nodes : T.cap_nodes;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nn;
         a += (int64_t)gridDim.x * blockDim.x) {
        const double M = T.M[a];
        const double r = M > 0.0 ? 1.0 / M : 0.0;
        ncot[3 * a] *= r;
        ncot[3 * a + 1] *= r;
        ncot[3 * a + 2] *= r;
    }
}

__global__ void k_leaf_sum(TreeDev T, double *q, int32_t *leaf_of)
{
    const int64_t nn = *T.n_nodes < T.cap_nodes ? *T.n_nodes : T.cap_nodes;
    if (*T.status == TP_ERR_LIST_OVERFLOW) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (T.nchild[i] != 0 || T.count[i] == 0) continue;
        int32_t chain[TP_NLEVELS];
        int d = 0;
        for (int32_t a = (int32_t)i; a >= 0 && d < TP_NLEVELS; a = T.parent[a]) chain[d++] = a;
        double Px = 0.0, Py = 0.0, Pz = 0.0;
        for (int k = d - 1; k >= 0; k--) {
            const int64_t a = chain[k];
            Px += q[3 * a];
            Py += q[3 * a + 1];
            Pz += q[3 * a + 2];
        }
        q[3 * i] = Px;
        q[3 * i + 1] = Py;
        q[3 * i + 2] = Pz;
        const int32_t f = T.first[i], e = f + T.count[i];
        for (int32_t p = f; p < e; p++) leaf_of[p] = (int32_t)i;
    }
}

__global__ void k_unsort_grad(TreeDev T, const double *gs, const double *P, const int32_t *leaf_of, double *grad)
{
    // after an overflow the leaves may not cover every particle: zeros, as the pair sums are
    const bool zero = *T.status == TP_ERR_LIST_OVERFLOW;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < T.n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = T.perm[s];
        if (zero) {
            grad[3 * o] = grad[3 * o + 1] = grad[3 * o + 2] = 0.0;
            continue;
        }
        const int64_t L = leaf_of[s];
        const BoxPrm &B = T.box[T.nbox > 1 ? tp_box_of(T.box_off, T.nbox, o) : 0];
        const double gk3 = B.gk2 * (2.0 / B.rcut), mp = T.m[s];
        grad[3 * o] = gk3 * (gs[3 * s] + mp * P[3 * L]);
        grad[3 * o + 1] = gk3 * (gs[3 * s + 1] + mp * P[3 * L + 1]);
        grad[3 * o + 2] = gk3 * (gs[3 * s + 2] + mp * P[3 * L + 2]);
    }
}

// Useful pairs (tp_stats.n_useful): the (group particle, list entry) pairs at
// a positive distance whose cutoff distance -- r, or s = sqrt(r^2 + eps^2)
// with the softened cutoff argument -- is below r_cut, so that their Eq. 2
// term is not identically zero.  The decision is the FP64 one of the
// definition: d = x_j - x_i from the FP64 positions (centres of mass for
// monopoles), reduced to the minimum image, r^2 = (dx dx + dy dy) + dz dz
// with every product and sum rounded separately, compared with r_cut^2.  An
// FP32 estimate of |d'|^2 from the entry records (scaled by k = 2/r_cut)
// settles every pair that lies clear of both thresholds (0 and the cutoff) by
// more than its error bound; the few others take the FP64 test.
__device__ __forceinline__ bool useful_f64(const TreeDev &T, const BoxPrm &P, int32_t i, int32_t e)
{
    double xj, yj, zj;
    if (e >= 0) {
        xj = T.x[e]; yj = T.y[e]; zj = T.z[e];
    } else {
        const int32_t nd = -e - 1;
        xj = T.comx[nd]; yj = T.comy[nd]; zj = T.comz[nd];
    }
    double dx = __dsub_rn(xj, T.x[i]), dy = __dsub_rn(yj, T.y[i]), dz = __dsub_rn(zj, T.z[i]);
    dx = __dsub_rn(dx, rint(dx));
    dy = __dsub_rn(dy, rint(dy));
    dz = __dsub_rn(dz, rint(dz));
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 == 0.0) return false;
    const double c2 = T.xi_soft ? __dadd_rn(r2, P.eps2) : r2;
    return c2 < P.rc2;
}

__global__ void __launch_bounds__(kThreads) k_count_useful(TreeDev T, unsigned long long *useful)
{
    __shared__ float px[kThreads], py[kThreads], pz[kThreads];
    const int64_t G_n = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    unsigned long long cnt = 0;
    if (*T.status != TP_ERR_LIST_OVERFLOW) {
        for (int64_t g = blockIdx.x; g < G_n; g += gridDim.x) {
            const Group G = load_group(T, g);
            const BoxPrm &P = *G.P;
            const float sc = P.scale, e2 = T.xi_soft ? P.eps2s : 0.f;
            // Offsets are at most H = k (h + r_cut) per axis (entries lie within
            // r_cut of the group box) and carry two FP32 roundings each (2.4e-7 H
            // per component of d'), so the estimate of |d'|^2 is off by at most
            // ~1.7e-6 H + 1e-6 near the cutoff (|d'| = 2), and a true |d'|^2 > 0
            // cannot round to 0 unless it is below ~1e-12 H^2; tol and tol0 keep
            // a margin of five or more over those.
            const double hm = fmax(T.ghx[g], fmax(T.ghy[g], T.ghz[g]));
            const float H = (float)((hm + P.rcut) * (2.0 / P.rcut));
            const float tol = 1e-5f * (H + 1.f), tol0 = 1e-10f * (H + 1.f) * (H + 1.f);
            for (int i0 = 0; i0 < G.ni; i0 += kThreads) {
                const int nic = min(kThreads, G.ni - i0);
                __syncthreads();
                if (threadIdx.x < nic) {
                    const int32_t p = G.first + i0 + threadIdx.x;
                    px[threadIdx.x] = Arith<float>::from_fixed(T.X[p], G.X, sc);
                    py[threadIdx.x] = Arith<float>::from_fixed(T.Y[p], G.Y, sc);
                    pz[threadIdx.x] = Arith<float>::from_fixed(T.Z[p], G.Z, sc);
                }
                __syncthreads();
                for (int q = threadIdx.x; q < G.ne; q += kThreads) {
                    const float4 r = T.rec[G.e0 + q];
                    const int32_t e = T.ent[G.e0 + q];
                    for (int k = 0; k < nic; k++) {
                        const int32_t i = G.first + i0 + k;
                        bool u;
                        if (G.wrap) {
                            u = useful_f64(T, P, i, e);
                        } else {
                            const float dx = r.x - px[k], dy = r.y - py[k], dz = r.z - pz[k];
                            const float r2 = dx * dx + dy * dy + dz * dz, c2 = r2 + e2;
                            u = (r2 > tol0 && fabsf(c2 - 4.f) > tol) ? c2 < 4.f : useful_f64(T, P, i, e);
                        }
                        cnt += u ? 1ull : 0ull;
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(useful, cnt);
}

// Launchers, instantiated for the plain (SOFT = false) and the softened
// (SOFT = true) cutoff argument; the tp:: entry points pick one per tree.
// The optional timing events bracket the pair kernel.  Under stream capture
// they are recorded as external events, which become event nodes of the
// graph, so each replay times the kernel too; otherwise as plain records.
void record_timing_event(cudaEvent_t ev, cudaStream_t s)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}
using tp::num_sms;
using tp::occupancy;

// One configuration of the packed forward kernel, on its own occupancy.
template <int NI, int TS, bool SOFT, bool RF>
void launch_pair_packed_rf(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s)
{
    static const int nb = occupancy(k_pair_packed<NI, TS, SOFT, RF>, kThreads);
    int64_t gr = (int64_t)num_sms() * nb;
    auto kp = k_pair_packed<NI, TS, SOFT, RF>;
    TP_LAUNCH(kp, (int)(gr > G ? G : gr), kThreads, 0, s, T, acc, queue, order);
}

template <int NI, int TS, bool SOFT>
void launch_pair_packed(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s)
{
    if (T.rsq_refined)
        launch_pair_packed_rf<NI, TS, SOFT, true>(T, acc, queue, order, G, s);
    else
        launch_pair_packed_rf<NI, TS, SOFT, false>(T, acc, queue, order, G, s);
}

template <bool SOFT>
void pair_forward_f32_t(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G,
                        cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int fwd_particles)
{
    cudaMemsetAsync(queue, 0, 2 * sizeof(int32_t), s);
    static const int bps = occupancy(k_pair<float, true, SOFT>, kThreads);
    if (ev0) record_timing_event(ev0, s);
    if (fwd_particles == 1)
        launch_pair_packed<1, 8, SOFT>(T, acc, queue + 1, order, G, s);
    else if (fwd_particles == 4)
        launch_pair_packed<4, 8, SOFT>(T, acc, queue + 1, order, G, s);
    else
        launch_pair_packed<2, 8, SOFT>(T, acc, queue + 1, order, G, s);
    if (ev1) record_timing_event(ev1, s);
    const int64_t gr = (int64_t)num_sms() * bps;
    auto k = k_pair<float, true, SOFT>;
    TP_LAUNCH(k, (int)(gr > G ? G : gr), kThreads, 0, s, T, acc, queue, order);
}

// The fused adjoint kernel with E entries per thread, with or without the
// forward sum, on its own occupancy.  E = 8 takes the entry-packed kernel
// (four pairs of entries per thread) for the forces and adjoint in one pass,
// and four entries per thread for the adjoint alone, whose four particle-side
// quantities gain less from the packing than the one pass's seven (measured:
// one pass 16.67 -> 16.47 ms on the clustered 2M box and 25.3 -> 23.1 ms in
// the paper regime; the adjoint alone 14.5 -> 15.4 and 20.0 -> 22.7 ms).
template <int E, bool SOFT, bool RF>
void launch_vjp_fused_rf(TreeDev &T, const float *cot, double *gs, double *ncot, int32_t *queue,
                         const int32_t *order, int64_t G, float *acc, cudaStream_t s)
{
    auto grid_of = [&](int per_sm) {
        int64_t gr = (int64_t)num_sms() * per_sm;
        return (int)(gr > G ? G : gr);
    };
    if (E == 8 && acc) {
        static const int nbw = occupancy(k_vjp_epack<4, true, SOFT, RF>, kThreads);
        auto kw = k_vjp_epack<4, true, SOFT, RF>;
        TP_LAUNCH(kw, grid_of(nbw), kThreads, 0, s, T, cot, gs, ncot, queue, order, acc);
        return;
    }
    constexpr int EF = E == 8 ? 4 : E;
    static const int nbf = occupancy(k_vjp_fused<EF, false, SOFT, RF>, kThreads);
    static const int nbw = occupancy(k_vjp_fused<EF, true, SOFT, RF>, kThreads);
    if (acc) {
        auto kw = k_vjp_fused<EF, true, SOFT, RF>;
        TP_LAUNCH(kw, grid_of(nbw), kThreads, 0, s, T, cot, gs, ncot, queue, order, acc);
    } else {
        auto kf = k_vjp_fused<EF, false, SOFT, RF>;
        TP_LAUNCH(kf, grid_of(nbf), kThreads, 0, s, T, cot, gs, ncot, queue, order, nullptr);
    }
}

template <int E, bool SOFT>
void launch_vjp_fused(TreeDev &T, const float *cot, double *gs, double *ncot, int32_t *queue,
                      const int32_t *order, int64_t G, float *acc, cudaStream_t s)
{
    if (T.rsq_refined)
        launch_vjp_fused_rf<E, SOFT, true>(T, cot, gs, ncot, queue, order, G, acc, s);
    else
        launch_vjp_fused_rf<E, SOFT, false>(T, cot, gs, ncot, queue, order, G, acc, s);
}

template <class R, bool SOFT>
void vjp_pairs_t(TreeDev &T, const R *cot, double *gs, double *ncot, int32_t *queue, const int32_t *order,
                 int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, float *acc, int adj_entries)
{
    static const int nb = occupancy(k_vjp<R, SOFT>, kThreads);
    auto grid_of = [&](int per_sm) {
        int64_t gr = (int64_t)num_sms() * per_sm;
        return (int)(gr > G ? G : gr);
    };
    if (sizeof(R) == 4) {
        cudaMemsetAsync(queue, 0, 2 * sizeof(int32_t), s);
        if (ev0) record_timing_event(ev0, s);
        if (adj_entries == 2)
            launch_vjp_fused<2, SOFT>(T, (const float *)cot, gs, ncot, queue + 1, order, G, acc, s);
        else if (adj_entries == 8)
            launch_vjp_fused<8, SOFT>(T, (const float *)cot, gs, ncot, queue + 1, order, G, acc, s);
        else
            launch_vjp_fused<4, SOFT>(T, (const float *)cot, gs, ncot, queue + 1, order, G, acc, s);
        if (ev1) record_timing_event(ev1, s);
    } else {
        cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
    }
    auto k = k_vjp<R, SOFT>;
    TP_LAUNCH(k, grid_of(nb), kThreads, 0, s, T, cot, gs, ncot, queue, order);
}

template <class R>
void vjp_pairs(TreeDev &T, const R *cot, double *gs, double *ncot, int32_t *queue, const int32_t *order,
               int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, float *acc = nullptr,
               int adj_entries = 4)
{
    if (G <= 0) return;
    if (T.xi_soft)
        vjp_pairs_t<R, true>(T, cot, gs, ncot, queue, order, G, s, ev0, ev1, acc, adj_entries);
    else
        vjp_pairs_t<R, false>(T, cot, gs, ncot, queue, order, G, s, ev0, ev1, acc, adj_entries);
}

// The general FP32 forward kernel for the groups the fused adjoint leaves.
template <bool SOFT>
void pair_rest_f32_t(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s)
{
    static const int bps = occupancy(k_pair<float, true, SOFT>, kThreads);
    const int64_t gr = (int64_t)num_sms() * bps;
    cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
    auto k = k_pair<float, true, SOFT>;
    TP_LAUNCH(k, (int)(gr > G ? G : gr), kThreads, 0, s, T, acc, queue, order);
}

}  // namespace

namespace tp {

// Queried once per process (thread-safe static initialisation), outside any
// stream capture: the first call of each launcher is never captured.
int num_sms()
{
    static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }();
    return sms;
}

void pair_forward_f32(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G,
                      cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int fwd_particles)
{
    if (G <= 0) return;
    if (T.xi_soft)
        pair_forward_f32_t<true>(T, acc, queue, order, G, s, ev0, ev1, fwd_particles);
    else
        pair_forward_f32_t<false>(T, acc, queue, order, G, s, ev0, ev1, fwd_particles);
}

void pair_forward_f64(TreeDev &T, double *acc, int64_t G, cudaStream_t s)
{
    if (G <= 0) return;
    int64_t grid = G < (1ll << 30) ? G : (1ll << 30);
    if (T.xi_soft) {
        auto k = k_pair<double, false, true>;
        TP_LAUNCH(k, (int)grid, kThreads, 0, s, T, acc, nullptr, nullptr);
    } else {
        auto k = k_pair<double, false, false>;
        TP_LAUNCH(k, (int)grid, kThreads, 0, s, T, acc, nullptr, nullptr);
    }
}

// The adjoint in three stages so that a caller can run the pair stage once
// per window of groups: zero the accumulators, the pair kernels, then the
// push-down of node cotangents and the scatter to input order.
void vjp_begin(TreeDev &T, double *gs, double *ncot, cudaStream_t s)
{
    cudaMemsetAsync(gs, 0, sizeof(double) * 3 * (size_t)T.n, s);
    cudaMemsetAsync(ncot, 0, sizeof(double) * 3 * (size_t)T.cap_nodes, s);
}

// leaf_of: scratch of n int32.
void vjp_end(TreeDev &T, double *grad, double *gs, double *ncot, int32_t *leaf_of, cudaStream_t s)
{
    if (T.n == 0) return;
    TP_LAUNCH(k_node_quot, grid_for(T.cap_nodes, 256), 256, 0, s, T, ncot);
    TP_LAUNCH(k_leaf_sum, grid_for(T.cap_nodes, 128), 128, 0, s, T, ncot, leaf_of);
    TP_LAUNCH(k_unsort_grad, grid_for(T.n, 256), 256, 0, s, T, gs, ncot, leaf_of, grad);
}

void vjp_pairs_f32(TreeDev &T, const float *cot, double *gs, double *ncot, int32_t *queue, const int32_t *order,
                   int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int adj_entries)
{
    vjp_pairs<float>(T, cot, gs, ncot, queue, order, G, s, ev0, ev1, nullptr, adj_entries);
}

// Forward and adjoint of the FP32 path in one pass over the lists: the fused
// adjoint kernel also sums Eq. 2 for the groups it takes; the general forward
// kernel covers the rest.  acc must be zeroed by the caller.
void force_vjp_pairs_f32(TreeDev &T, float *acc, const float *cot, double *gs, double *ncot, int32_t *queue,
                         const int32_t *order, int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                         int adj_entries)
{
    if (G <= 0) return;
    vjp_pairs<float>(T, cot, gs, ncot, queue, order, G, s, ev0, ev1, acc, adj_entries);
    if (T.xi_soft)
        pair_rest_f32_t<true>(T, acc, queue, order, G, s);
    else
        pair_rest_f32_t<false>(T, acc, queue, order, G, s);
}

// Useful-pair count of whole lists into *useful (zeroed by the caller).
void count_useful(TreeDev &T, unsigned long long *useful, cudaStream_t s)
{
    if (T.cap_groups <= 0) return;
    const int64_t gr = (int64_t)num_sms() * 8;
    TP_LAUNCH(k_count_useful, (int)(gr > T.cap_groups ? T.cap_groups : gr), kThreads, 0, s, T, useful);
}

void vjp_pairs_f64(TreeDev &T, const double *cot, double *gs, double *ncot, int32_t *queue,
                   const int32_t *order, int64_t G, cudaStream_t s)
{
    vjp_pairs<double>(T, cot, gs, ncot, queue, order, G, s, nullptr, nullptr);
}

void vjp_f32(TreeDev &T, const float *cot, double *grad, double *gs, double *ncot, int32_t *leaf_of,
             int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
             int adj_entries)
{
    vjp_begin(T, gs, ncot, s);
    vjp_pairs<float>(T, cot, gs, ncot, queue, order, G, s, ev0, ev1, nullptr, adj_entries);
    vjp_end(T, grad, gs, ncot, leaf_of, s);
}

void vjp_f64(TreeDev &T, const double *cot, double *grad, double *gs, double *ncot, int32_t *leaf_of,
             int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s)
{
    vjp_begin(T, gs, ncot, s);
    vjp_pairs<double>(T, cot, gs, ncot, queue, order, G, s, nullptr, nullptr);
    vjp_end(T, grad, gs, ncot, leaf_of, s);
}

}  // namespace tp
