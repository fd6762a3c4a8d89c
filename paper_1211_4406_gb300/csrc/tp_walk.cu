// tp_walk.cu -- per-group interaction lists (Barnes' modified algorithm,
// Sec. II; the "tree traversal" row of Table I).
//
// One thread walks one group's tree depth first, without a stack, by the skip
// pointers of the breadth-first node array.  At every node it decides
//   prune   periodic box-to-box gap d >= r_cut,
//   accept  no overlap with the group, largest box-to-box distance < r_cut and
//           l^2 < theta^2 d^2 (l = 2^-level): the node enters as a monopole,
//   open    otherwise (at a leaf: keep particles with point-to-box gap < r_cut).
// The decisions must equal the FP64 ones of the reference definition bit for
// bit.  GB300 runs FP64 at a small fraction of its FP32/integer rate, so each
// one is first taken on a 2^-32 integer grid: positions, centres and half-widths
// are truncated to 32-bit fixed point, wrap-around subtraction gives the
// periodic minimum image for free, and the squared gaps are exact 64-bit
// integers.  Truncation moves every gap by less than TP_FILTER_SLACK grid
// units, so comparing with thresholds widened by that slack either settles the
// decision for certain or, in a band of a few 1e-9 of the box, falls back to the
// same FP64 expression evaluated with round-to-nearest intrinsics.
#include "tp_common.cuh"

namespace {

constexpr int kBlock = 128;

__device__ __forceinline__ uint32_t absdiff32(uint32_t a, uint32_t b)
{
    const int32_t t = (int32_t)(a - b);
    return t < 0 ? (uint32_t)(-(int64_t)t) : (uint32_t)t;
}

__device__ __forceinline__ double dminimg(double t) { return __dsub_rn(t, rint(t)); }

// Reference FP64 box distances: per axis t = |minimg(a - c)|, s = h + hg,
// gap = max(0, t - s), far = t + s; sums (x^2 + y^2) + z^2.
__device__ __forceinline__ double exact_dist2(double ax, double ay, double az, double hx, double hy,
                                              double hz, double cx, double cy, double cz, double gx,
                                              double gy, double gz, double *far2)
{
    const double a[3] = {ax, ay, az}, h[3] = {hx, hy, hz}, c[3] = {cx, cy, cz}, g[3] = {gx, gy, gz};
    double gp[3], fr[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double tt = fabs(dminimg(__dsub_rn(a[k], c[k])));
        const double s = __dadd_rn(h[k], g[k]);
        const double e = __dsub_rn(tt, s);
        gp[k] = e > 0.0 ? e : 0.0;
        fr[k] = __dadd_rn(tt, s);
    }
    *far2 = __dadd_rn(__dadd_rn(__dmul_rn(fr[0], fr[0]), __dmul_rn(fr[1], fr[1])), __dmul_rn(fr[2], fr[2]));
    return __dadd_rn(__dadd_rn(__dmul_rn(gp[0], gp[0]), __dmul_rn(gp[1], gp[1])), __dmul_rn(gp[2], gp[2]));
}

template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_walk(TreeDev T, int64_t G_cap)
{
    const int64_t G = *T.n_groups < G_cap ? *T.n_groups : G_cap;
    if (WRITE && *T.status == TP_ERR_LIST_OVERFLOW) return;   // lists would not fit
    unsigned long long ambig = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = T.gbox[g];
        const BoxPrm &P = T.box[b];
        const uint32_t gx = T.gux[g], gy = T.guy[g], gz = T.guz[g];
        const uint32_t hx = T.ghux[g], hy = T.ghuy[g], hz = T.ghuz[g];
        const int32_t g0 = T.gfirst[g], g1 = g0 + T.gcount[g];
        const uint64_t T_lo = P.T_lo, T_hi = P.T_hi;
        int64_t out = WRITE ? T.loff[g] : 0;
        int64_t out_end = WRITE ? out + T.lcnt[g] : 0;
        if (WRITE && out_end > T.cap_entries) out_end = T.cap_entries;
        int32_t cnt = 0;
        int32_t nd = b;                       // the box root
        int64_t budget = *T.n_nodes + 1;      // a preorder walk visits each node at most once
        while (nd >= 0) {
            if (--budget < 0 || nd >= T.cap_nodes) {
                tp_latch(T.status, TP_ERR_TIMEOUT);
                break;
            }
            const WNode w = T.wn[nd];
            const uint32_t ax = absdiff32(w.cx, gx), ay = absdiff32(w.cy, gy), az = absdiff32(w.cz, gz);
            const uint64_t sx = (uint64_t)w.hx + hx, sy = (uint64_t)w.hy + hy, sz = (uint64_t)w.hz + hz;
            const uint64_t dx = ax > sx ? ax - sx : 0, dy = ay > sy ? ay - sy : 0, dz = az > sz ? az - sz : 0;
            const uint64_t gap2 = dx * dx + dy * dy + dz * dz;
            bool exact = false, prune;
            double gap2d = 0.0, far2d = 0.0;
            if (gap2 >= T_hi) {
                prune = true;
            } else if (gap2 < T_lo) {
                prune = false;
            } else {
                exact = true;
                ambig++;
                gap2d = exact_dist2(T.cenx[nd], T.ceny[nd], T.cenz[nd], T.hfx[nd], T.hfy[nd], T.hfz[nd],
                                    T.gcx[g], T.gcy[g], T.gcz[g], T.ghx[g], T.ghy[g], T.ghz[g], &far2d);
                prune = gap2d >= P.rc2;
            }
            if (prune) { nd = w.skip; continue; }
            const bool overlap = w.first < g1 && g0 < w.first + w.count;
            bool accept = false;
            if (!overlap) {
                if (!exact) {
                    const uint64_t fx = ax + sx, fy = ay + sy, fz = az + sz;
                    const uint64_t far2 = ((fx | fy | fz) >> 31) ? ~0ull : fx * fx + fy * fy + fz * fz;
                    const int A = far2 < T_lo ? 1 : (far2 >= T_hi ? 0 : -1);
                    const int B = gap2 >= P.TB_hi[w.level] ? 1 : (gap2 < P.TB_lo[w.level] ? 0 : -1);
                    if (A == 0 || B == 0) {
                        accept = false;
                    } else if (A == 1 && B == 1) {
                        accept = true;
                    } else {
                        exact = true;
                        ambig++;
                        gap2d = exact_dist2(T.cenx[nd], T.ceny[nd], T.cenz[nd], T.hfx[nd], T.hfy[nd],
                                            T.hfz[nd], T.gcx[g], T.gcy[g], T.gcz[g], T.ghx[g], T.ghy[g],
                                            T.ghz[g], &far2d);
                    }
                }
                if (exact) {
                    const double l = ldexp(1.0, -w.level);
                    accept = far2d < P.rc2 && __dmul_rn(l, l) < __dmul_rn(P.th2, gap2d);
                }
            }
            if (accept) {
                if (WRITE && out < out_end) T.ent[out++] = -(nd + 1);
                cnt++;
                nd = w.skip;
                continue;
            }
            if (w.child < 0) {
                for (int32_t p = w.first; p < w.first + w.count; p++) {
                    const uint32_t qx = absdiff32((uint32_t)(T.X[p] >> 32), gx);
                    const uint32_t qy = absdiff32((uint32_t)(T.Y[p] >> 32), gy);
                    const uint32_t qz = absdiff32((uint32_t)(T.Z[p] >> 32), gz);
                    const uint64_t ex = qx > hx ? qx - hx : 0, ey = qy > hy ? qy - hy : 0,
                                   ez = qz > hz ? qz - hz : 0;
                    const uint64_t p2 = ex * ex + ey * ey + ez * ez;
                    bool keep;
                    if (p2 >= T_hi) {
                        keep = false;
                    } else if (p2 < T_lo) {
                        keep = true;
                    } else {
                        ambig++;
                        double f2;
                        keep = exact_dist2(T.x[p], T.y[p], T.z[p], 0.0, 0.0, 0.0, T.gcx[g], T.gcy[g], T.gcz[g],
                                           T.ghx[g], T.ghy[g], T.ghz[g], &f2) < P.rc2;
                    }
                    if (keep) {
                        if (WRITE && out < out_end) T.ent[out++] = p;
                        cnt++;
                    }
                }
                nd = w.skip;
            } else {
                nd = w.child;
            }
        }
        if (!WRITE) T.lcnt[g] = cnt;
        else if (out != T.loff[g] + cnt) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
    }
    if (!WRITE && ambig) atomicAdd(T.n_ambig, ambig);
}

__global__ void k_list_stats(TreeDev T, unsigned long long *inter, int32_t *max_nj)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    unsigned long long s = 0;
    int32_t mx = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        s += (unsigned long long)T.gcount[g] * (unsigned long long)T.lcnt[g];
        mx = max(mx, T.lcnt[g]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(inter, s);
        atomicMax(max_nj, mx);
    }
}

}  // namespace

namespace tp {

void walk_count(TreeDev &T, int64_t G_cap, cudaStream_t s)
{
    if (G_cap <= 0) return;
    TP_LAUNCH(k_walk<false>, grid_for(G_cap, kBlock), kBlock, 0, s, T, G_cap);
}

void walk_write(TreeDev &T, int64_t G_cap, cudaStream_t s)
{
    if (G_cap <= 0) return;
    TP_LAUNCH(k_walk<true>, grid_for(G_cap, kBlock), kBlock, 0, s, T, G_cap);
}

void list_stats(TreeDev &T, unsigned long long *inter, int32_t *max_nj, cudaStream_t s)
{
    TP_LAUNCH(k_list_stats, 152 * 2, 256, 0, s, T, inter, max_nj);
}

}  // namespace tp
