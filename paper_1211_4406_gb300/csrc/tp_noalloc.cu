// tp_noalloc.cu -- tp_short_range_force_noalloc: the short-range acceleration
// of a small box without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: an application whose
// device memory is carved from its own pool and forbids other allocations, or
// a latency-critical loop where an allocation's implicit synchronisation is
// not acceptable.  For them this entry point keeps its scratch -- the 64-bit
// fixed-point images and the masses of the particles, and one status word --
// in one statically sized device array that the CUDA driver places when the
// library's module is loaded.  Every GPU that loads the library holds that
// array (28 bytes per particle x TP_NOALLOC_MAX_N = 1.8 MB) until the process
// exits.
//
// The sum is taken directly over all pairs (no tree): the exact cutoff sum,
// the same force as the tree path at theta = 0, up to FP32 rounding.  Each
// pair's minimum-image offset is the wrap-around difference of the two
// fixed-point images, converted once to FP32 and scaled by k = 2/r_cut; the
// cutoff function is evaluated in the cancellation-free form u^5 h(xi) +
// v^6 c(xi) used by the tree path; tile sums are accumulated in FP64.  A
// non-finite position is detected while the images are taken: the call then
// returns TP_ERR_NONFINITE (it synchronises its stream once for that) and
// leaves acc unwritten.  Every call fully rewrites the part of the scratch it
// reads and clears the status word first, so nothing has to be cleared
// between calls; calls that overlap on the GPU share the array and race.
#include <cmath>
#include <mutex>

#include "tp_common.cuh"

namespace {

constexpr int kNaThreads = 128;
constexpr size_t kNaBytes = (size_t)TP_NOALLOC_MAX_N * (3 * sizeof(uint64_t) + sizeof(float));

// Layout: X[max], Y[max], Z[max] (uint64), M[max] (float), then the status
// word (int32) of the last call.
static __device__ __align__(256) unsigned char tp_noalloc_scratch[kNaBytes + 256];

struct NaView {
    uint64_t *X, *Y, *Z;
    float *M;
    int32_t *status;
};

__host__ __device__ inline NaView na_view(unsigned char *base)
{
    NaView v;
    v.X = reinterpret_cast<uint64_t *>(base);
    v.Y = v.X + TP_NOALLOC_MAX_N;
    v.Z = v.Y + TP_NOALLOC_MAX_N;
    v.M = reinterpret_cast<float *>(v.Z + TP_NOALLOC_MAX_N);
    v.status = reinterpret_cast<int32_t *>(base + kNaBytes);
    return v;
}

__device__ __forceinline__ double na_wrap(double x)
{
    const double w = __dsub_rn(x, floor(x));
    return w >= 1.0 ? 0.0 : w;
}

__device__ __forceinline__ float na_sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__global__ void k_na_images(const double *pos, const double *mass, int n, float inv_n, NaView S)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = pos[3 * (int64_t)i], y = pos[3 * (int64_t)i + 1], z = pos[3 * (int64_t)i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
            // no image of a non-finite coordinate exists: record the error
            // (the host refuses the call) and write a defined value
            atomicCAS(S.status, 0, (int32_t)TP_ERR_NONFINITE);
            S.X[i] = S.Y[i] = S.Z[i] = 0ull;
        } else {
            S.X[i] = tp_fixed64(na_wrap(x));
            S.Y[i] = tp_fixed64(na_wrap(y));
            S.Z[i] = tp_fixed64(na_wrap(z));
        }
        S.M[i] = mass ? (float)mass[i] : inv_n;
    }
}

__global__ void __launch_bounds__(kNaThreads) k_na_pairs(NaView S, int n, float sc, float eps2, double gk2,
                                                         float *acc)
{
    __shared__ uint64_t sx[kNaThreads], sy[kNaThreads], sz[kNaThreads];
    __shared__ float sm[kNaThreads];
    for (int i0 = blockIdx.x * kNaThreads; i0 < n; i0 += gridDim.x * kNaThreads) {
        const int i = i0 + threadIdx.x;
        const bool vi = i < n;
        const uint64_t xi = vi ? S.X[i] : 0, yi = vi ? S.Y[i] : 0, zi = vi ? S.Z[i] : 0;
        double sax = 0.0, say = 0.0, saz = 0.0;
        for (int j0 = 0; j0 < n; j0 += kNaThreads) {
            __syncthreads();
            const int j = j0 + threadIdx.x;
            if (j < n) {
                sx[threadIdx.x] = S.X[j]; sy[threadIdx.x] = S.Y[j]; sz[threadIdx.x] = S.Z[j];
                sm[threadIdx.x] = S.M[j];
            }
            __syncthreads();
            const int nt = min(kNaThreads, n - j0);
            float ax = 0.f, ay = 0.f, az = 0.f;
            if (vi) {
                for (int q = 0; q < nt; q++) {
                    const float dx = __ll2float_rn((long long)(sx[q] - xi)) * sc;
                    const float dy = __ll2float_rn((long long)(sy[q] - yi)) * sc;
                    const float dz = __ll2float_rn((long long)(sz[q] - zi)) * sc;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float ri = rsqrtf(r2 + eps2);
                    const float x = na_sqrt_approx(r2);
                    const float u = fmaxf(2.f - x, 0.f), v = fmaxf(1.f - x, 0.f);
                    float h = (7.f / 140.f) * x + 22.f / 140.f;
                    h = h * x + 10.f / 140.f;
                    h = h * x + 4.f / 140.f;
                    float c = (7.f / 35.f) * x + 18.f / 35.f;
                    c = c * x + 3.f / 35.f;
                    const float u2 = u * u, v2 = v * v;
                    const float g = (v2 * v2 * v2) * c + (u2 * u2 * u) * h;
                    float f = sm[q] * g * (ri * ri * ri);
                    f = r2 > 0.f ? f : 0.f;          // the particle itself, coincident pairs
                    ax += f * dx;
                    ay += f * dy;
                    az += f * dz;
                }
            }
            sax += ax; say += ay; saz += az;
        }
        if (vi) {
            acc[3 * (int64_t)i] = (float)(sax * gk2);
            acc[3 * (int64_t)i + 1] = (float)(say * gk2);
            acc[3 * (int64_t)i + 2] = (float)(saz * gk2);
        }
    }
}

// Device (or managed) memory that belongs to the current device: the kernels
// run there and must not read another GPU's memory through this path.
bool na_is_device_ptr(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch array, looked up once per device (host code
// cannot use the array's name as a device pointer) and kept for the life of
// the process; a cudaDeviceReset unloads the module, so the cached address
// does not survive one.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char *g_na_ptr[kNaMaxDevices] = {};

tp_status na_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kNaMaxDevices) return TP_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, tp_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return TP_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_ptr[dev];
    return TP_OK;
}

}  // namespace

extern "C" tp_status tp_short_range_force_noalloc(const double *pos, const double *mass, int64_t n,
                                                  const tp_params *p, float *acc, void *stream)
{
    if (!p || n < 0 || n > TP_NOALLOC_MAX_N) return TP_ERR_INVALID_ARG;
    if (!(p->r_cut > 0.0 && p->r_cut < 0.5) || !(p->eps >= 0.0) || !std::isfinite(p->eps) ||
        !std::isfinite(p->G) || p->precision != TP_FP32 || p->flags != 0)
        return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return TP_ERR_NO_DEVICE;
    }
    if (!na_is_device_ptr(pos, dev) || !na_is_device_ptr(acc, dev) || (mass && !na_is_device_ptr(mass, dev)))
        return TP_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    const tp_status st = na_scratch(dev, &base);
    if (st != TP_OK) return st;
    const NaView S = na_view(base);
    const double k = 2.0 / p->r_cut;
    const float sc = (float)(k * 5.421010862427522e-20);      // k * 2^-64
    const float eps2 = (float)((k * p->eps) * (k * p->eps));
    const double gk2 = p->G * k * k;
    const int ni = (int)n;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (ni + kNaThreads - 1) / kNaThreads;
    if (cudaMemsetAsync(S.status, 0, sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return TP_ERR_CUDA;
    }
    TP_LAUNCH(k_na_images, blocks, kNaThreads, 0, s, pos, mass, ni, (float)(1.0 / (double)n), S);
    // the status of the positions, read back before the pair sum is enqueued
    int32_t status = 0;
    if (cudaMemcpyAsync(&status, S.status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TP_ERR_CUDA;
    }
    if (status != 0) return (tp_status)status;
    TP_LAUNCH(k_na_pairs, blocks, kNaThreads, 0, s, S, ni, sc, eps2, gk2, acc);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}
