// tp_pm.cu -- the long-range (PM) half of TreePM (the density split of
// Sec. II, the PM cycle of Sec. II-B): the cycle the paper runs every step,
// on one GPU and an N^3 periodic mesh of the unit box.
//
//   k_pm_assign   TSC mass assignment: each particle adds its mass to the 27
//                 mesh points around its nearest one (FP32 atomics, L2)
//   cuFFT R2C     forward transform of the mass per cell
//   k_pm_green    product with the Green's function of the long-range force
//   cuFFT C2R     back to the potential on the mesh
//   k_pm_gradient four-point difference of the potential, -grad(phi), written
//                 as one float4 per cell so the interpolation reads 16 bytes
//   k_pm_interp   TSC interpolation of the mesh force to each particle
//
// Mesh point (i, j, k) sits at (i h, j h, k h), h = 1/N, stored at
// (i N + j) N + k.  The long-range pair force is the force between two S2
// clouds of radius r_cut/2 (Eq. 1), so the Green's function is
// -4 pi G S(k)^2 / k^2 with S(x) = 12 (2 - 2 cos x - x sin x) / x^4 at
// x = k r_cut / 2, divided by the square of the TSC window (assignment and
// interpolation) and zero at k = 0.  With the mass per cell on the mesh
// (not the density) and cuFFT's unnormalised inverse, the factors h^-3 and
// N^-3 cancel, so the table holds exactly that function.
#include <cufft.h>

#include <cmath>
#include <new>

#include "tp_common.cuh"
#include "tp_nvtx.h"

namespace {

constexpr int kPmThreads = 256;

__device__ __forceinline__ double pm_wrap(double x)
{
    double w = x - floor(x);
    return w >= 1.0 ? 0.0 : w;
}

// Nearest mesh point of one coordinate and its three TSC weights (offsets
// -1, 0, +1).
__device__ __forceinline__ void tsc(double x, int N, int &i0, float w[3])
{
    const double u = pm_wrap(x) * N;
    const double c = rint(u);
    const double d = u - c;
    i0 = (int)c;
    const double a = 0.5 - d, b = 0.5 + d;
    w[0] = (float)(0.5 * a * a);
    w[1] = (float)(0.75 - d * d);
    w[2] = (float)(0.5 * b * b);
}

__device__ __forceinline__ int wrapi(int i, int N) { return i < 0 ? i + N : (i >= N ? i - N : i); }

__global__ void k_pm_assign(const double *pos, const double *mass, int64_t n, int N, float m_default,
                            float *rho)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float wx[3], wy[3], wz[3];
        tsc(pos[3 * p], N, ix, wx);
        tsc(pos[3 * p + 1], N, iy, wy);
        tsc(pos[3 * p + 2], N, iz, wz);
        const float m = mass ? (float)mass[p] : m_default;
        for (int a = 0; a < 3; a++) {
            const int64_t ra = (int64_t)wrapi(ix + a - 1, N) * N;
            const float ma = m * wx[a];
            for (int b = 0; b < 3; b++) {
                const int64_t rb = (ra + wrapi(iy + b - 1, N)) * N;
                const float mb = ma * wy[b];
                for (int c = 0; c < 3; c++) atomicAdd(rho + rb + wrapi(iz + c - 1, N), mb * wz[c]);
            }
        }
    }
}

// Unit-mass S2 transform at x = k r_cut / 2; the Taylor series to x^8 below
// x = 0.3, where the closed form's bracket (~x^4/12) cancels.
__device__ double s2_hat(double x)
{
    if (x < 0.3) {
        const double x2 = x * x;
        return 1.0 + x2 * (-1.0 / 15.0 + x2 * (1.0 / 560.0 + x2 * (-1.0 / 37800.0 + x2 / 3991680.0)));
    }
    double s, c;
    sincos(x, &s, &c);
    const double x2 = x * x;
    return 12.0 * (2.0 - 2.0 * c - x * s) / (x2 * x2);
}

__device__ __forceinline__ double sinc_half(double k, double h)
{
    const double t = 0.5 * k * h;
    return t == 0.0 ? 1.0 : sin(t) / t;
}

__global__ void k_pm_green_table(float *green, int N, double r_cut, double G)
{
    const int Nz = N / 2 + 1;
    const int64_t total = (int64_t)N * N * Nz;
    const double h = 1.0 / N, twopi = 6.283185307179586476925;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(q % Nz);
        const int ky = (int)((q / Nz) % N);
        const int kx = (int)(q / ((int64_t)Nz * N));
        const double fx = twopi * (kx < (N + 1) / 2 ? kx : kx - N);
        const double fy = twopi * (ky < (N + 1) / 2 ? ky : ky - N);
        const double fz = twopi * kz;
        const double k2 = fx * fx + fy * fy + fz * fz;
        if (k2 == 0.0) {
            green[q] = 0.0f;
            continue;
        }
        const double s = s2_hat(sqrt(k2) * 0.5 * r_cut);
        const double w = sinc_half(fx, h) * sinc_half(fy, h) * sinc_half(fz, h);
        const double w3 = w * w * w;
        green[q] = (float)(-4.0 * 3.14159265358979323846 * G * s * s / (k2 * w3 * w3));
    }
}

__global__ void k_pm_green(cufftComplex *spec, const float *green, int64_t total)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float g = green[q];
        cufftComplex v = spec[q];
        v.x *= g;
        v.y *= g;
        spec[q] = v;
    }
}

// -grad(phi) by the four-point difference (8 (P[+1] - P[-1]) - (P[+2] - P[-2])) / 12h.
__global__ void k_pm_gradient(const float *phi, float4 *amesh, int N)
{
    const int64_t total = (int64_t)N * N * N;
    const float s = -(float)N / 12.0f;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q % N);
        const int j = (int)((q / N) % N);
        const int i = (int)(q / ((int64_t)N * N));
        auto P = [&](int a, int b, int c) {
            return phi[((int64_t)wrapi(a, N) * N + wrapi(b, N)) * N + wrapi(c, N)];
        };
        float4 r;
        r.x = s * (8.0f * (P(i + 1, j, k) - P(i - 1, j, k)) - (P(i + 2, j, k) - P(i - 2, j, k)));
        r.y = s * (8.0f * (P(i, j + 1, k) - P(i, j - 1, k)) - (P(i, j + 2, k) - P(i, j - 2, k)));
        r.z = s * (8.0f * (P(i, j, k + 1) - P(i, j, k - 1)) - (P(i, j, k + 2) - P(i, j, k - 2)));
        r.w = 0.0f;
        amesh[q] = r;
    }
}

__global__ void k_pm_interp(const double *pos, int64_t n, int N, const float4 *amesh, float *acc, int accumulate)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float wx[3], wy[3], wz[3];
        tsc(pos[3 * p], N, ix, wx);
        tsc(pos[3 * p + 1], N, iy, wy);
        tsc(pos[3 * p + 2], N, iz, wz);
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int a = 0; a < 3; a++) {
            const int64_t ra = (int64_t)wrapi(ix + a - 1, N) * N;
            for (int b = 0; b < 3; b++) {
                const int64_t rb = (ra + wrapi(iy + b - 1, N)) * N;
                const float wab = wx[a] * wy[b];
                for (int c = 0; c < 3; c++) {
                    const float4 v = __ldg(amesh + rb + wrapi(iz + c - 1, N));
                    const float w = wab * wz[c];
                    ax = fmaf(w, v.x, ax);
                    ay = fmaf(w, v.y, ay);
                    az = fmaf(w, v.z, az);
                }
            }
        }
        if (accumulate) {
            acc[3 * p] += ax;
            acc[3 * p + 1] += ay;
            acc[3 * p + 2] += az;
        } else {
            acc[3 * p] = ax;
            acc[3 * p + 1] = ay;
            acc[3 * p + 2] = az;
        }
    }
}

// ---------------------------------------------------------------------------
// The adjoint of the PM cycle.  For L = sum_i w_i . a_i:
//   dL/dx_k = sum_c grad W_k(c) [w_k . A(c) + m_k B(c)]
// with A = -grad(phi) the mesh force, U the TSC assignment of the cotangent
// vectors, and B = K div(U): the same potential solve K (symmetric: a real,
// even Green's function) applied to the four-point divergence of U (the
// four-point difference is antisymmetric, so it is its own transpose up to
// sign).  grad W_k is the derivative of particle k's weight at c.
// ---------------------------------------------------------------------------
__global__ void k_pm_assign_vec(const double *pos, const float *cot, int64_t n, int N, float4 *umesh)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float wx[3], wy[3], wz[3];
        tsc(pos[3 * p], N, ix, wx);
        tsc(pos[3 * p + 1], N, iy, wy);
        tsc(pos[3 * p + 2], N, iz, wz);
        const float cx = cot[3 * p], cy = cot[3 * p + 1], cz = cot[3 * p + 2];
        for (int a = 0; a < 3; a++) {
            const int64_t ra = (int64_t)wrapi(ix + a - 1, N) * N;
            for (int b = 0; b < 3; b++) {
                const int64_t rb = (ra + wrapi(iy + b - 1, N)) * N;
                const float wab = wx[a] * wy[b];
                for (int c = 0; c < 3; c++) {
                    float *u = reinterpret_cast<float *>(umesh + rb + wrapi(iz + c - 1, N));
                    const float w = wab * wz[c];
                    atomicAdd(u, w * cx);
                    atomicAdd(u + 1, w * cy);
                    atomicAdd(u + 2, w * cz);
                }
            }
        }
    }
}

// div(U) by the four-point difference along each axis.
__global__ void k_pm_divergence(const float4 *umesh, float *out, int N)
{
    const int64_t total = (int64_t)N * N * N;
    const float s = (float)N / 12.0f;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q % N);
        const int j = (int)((q / N) % N);
        const int i = (int)(q / ((int64_t)N * N));
        auto U = [&](int a, int b, int c) { return umesh[((int64_t)wrapi(a, N) * N + wrapi(b, N)) * N + wrapi(c, N)]; };
        const float dx = 8.0f * (U(i + 1, j, k).x - U(i - 1, j, k).x) - (U(i + 2, j, k).x - U(i - 2, j, k).x);
        const float dy = 8.0f * (U(i, j + 1, k).y - U(i, j - 1, k).y) - (U(i, j + 2, k).y - U(i, j - 2, k).y);
        const float dz = 8.0f * (U(i, j, k + 1).z - U(i, j, k - 1).z) - (U(i, j, k + 2).z - U(i, j, k - 2).z);
        out[q] = s * (dx + dy + dz);
    }
}

// B (the potential solve of div U, in bmesh) into the w lane of the force mesh.
__global__ void k_pm_pack_w(float4 *amesh, const float *bmesh, int64_t total)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        amesh[q].w = bmesh[q];
}

__device__ __forceinline__ void tsc_d(double x, int N, int &i0, float w[3], float dw[3])
{
    const double u = pm_wrap(x) * N;
    const double c = rint(u);
    const double d = u - c;
    i0 = (int)c;
    const double a = 0.5 - d, b = 0.5 + d;
    w[0] = (float)(0.5 * a * a);
    w[1] = (float)(0.75 - d * d);
    w[2] = (float)(0.5 * b * b);
    dw[0] = (float)(-a * N);
    dw[1] = (float)(-2.0 * d * N);
    dw[2] = (float)(b * N);
}

__global__ void k_pm_vjp_interp(const double *pos, const double *mass, float m_default, const float *cot, int64_t n,
                                int N, const float4 *amesh, double *grad, int accumulate)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        float wx[3], wy[3], wz[3], dx[3], dy[3], dz[3];
        tsc_d(pos[3 * p], N, ix, wx, dx);
        tsc_d(pos[3 * p + 1], N, iy, wy, dy);
        tsc_d(pos[3 * p + 2], N, iz, wz, dz);
        const float cx = cot[3 * p], cy = cot[3 * p + 1], cz = cot[3 * p + 2];
        const float m = mass ? (float)mass[p] : m_default;
        float gx = 0.f, gy = 0.f, gz = 0.f;
        for (int a = 0; a < 3; a++) {
            const int64_t ra = (int64_t)wrapi(ix + a - 1, N) * N;
            for (int b = 0; b < 3; b++) {
                const int64_t rb = (ra + wrapi(iy + b - 1, N)) * N;
                for (int c = 0; c < 3; c++) {
                    const float4 v = __ldg(amesh + rb + wrapi(iz + c - 1, N));
                    const float sv = fmaf(cx, v.x, fmaf(cy, v.y, fmaf(cz, v.z, m * v.w)));
                    gx = fmaf(dx[a] * wy[b] * wz[c], sv, gx);
                    gy = fmaf(wx[a] * dy[b] * wz[c], sv, gy);
                    gz = fmaf(wx[a] * wy[b] * dz[c], sv, gz);
                }
            }
        }
        if (accumulate) {
            grad[3 * p] += gx;
            grad[3 * p + 1] += gy;
            grad[3 * p + 2] += gz;
        } else {
            grad[3 * p] = gx;
            grad[3 * p + 1] = gy;
            grad[3 * p + 2] = gz;
        }
    }
}

bool is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int pm_grid(int64_t work, int block)
{
    const int64_t g = (work + block - 1) / block;
    const int64_t cap = (int64_t)tp::num_sms() * 16;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

struct tp_pm {
    int N = 0;
    double r_cut = 0.0, G = 0.0;
    float *rho = nullptr;           // [N^3] mass per cell, then (in place of it) the potential
    cufftComplex *spec = nullptr;   // [N][N][N/2+1]
    float *green = nullptr;         // [N][N][N/2+1]
    float4 *amesh = nullptr;        // [N^3] -grad(phi); w: the adjoint's B
    float4 *umesh = nullptr;        // [N^3] assigned cotangent vectors (adjoint; allocated on first use)
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
};

static void pm_release(tp_pm *pm)
{
    if (!pm) return;
    if (pm->have_fwd) cufftDestroy(pm->fwd);
    if (pm->have_inv) cufftDestroy(pm->inv);
    cudaFree(pm->rho);
    cudaFree(pm->spec);
    cudaFree(pm->green);
    cudaFree(pm->amesh);
    cudaFree(pm->umesh);
    delete pm;
}

extern "C" tp_status tp_pm_create(int32_t n_mesh, double r_cut, double G, void *stream, tp_pm **out)
{
    if (!out) return TP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_mesh < 8 || n_mesh > 1024 || (n_mesh & 1)) return TP_ERR_INVALID_ARG;
    if (!(r_cut > 0.0 && r_cut < 0.5) || !std::isfinite(G)) return TP_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return TP_ERR_NO_DEVICE;
    }
    tp_pm *pm = new (std::nothrow) tp_pm();
    if (!pm) return TP_ERR_OOM;
    pm->N = n_mesh;
    pm->r_cut = r_cut;
    pm->G = G;
    const int64_t N = n_mesh, cells = N * N * N, half = N * N * (N / 2 + 1);
    if (cudaMalloc(&pm->rho, sizeof(float) * cells) != cudaSuccess ||
        cudaMalloc(&pm->spec, sizeof(cufftComplex) * half) != cudaSuccess ||
        cudaMalloc(&pm->green, sizeof(float) * half) != cudaSuccess ||
        cudaMalloc(&pm->amesh, sizeof(float4) * cells) != cudaSuccess) {
        cudaGetLastError();
        pm_release(pm);
        return TP_ERR_OOM;
    }
    if (cufftPlan3d(&pm->fwd, n_mesh, n_mesh, n_mesh, CUFFT_R2C) != CUFFT_SUCCESS) {
        pm_release(pm);
        return TP_ERR_CUDA;
    }
    pm->have_fwd = true;
    if (cufftPlan3d(&pm->inv, n_mesh, n_mesh, n_mesh, CUFFT_C2R) != CUFFT_SUCCESS) {
        pm_release(pm);
        return TP_ERR_CUDA;
    }
    pm->have_inv = true;
    cudaStream_t s = (cudaStream_t)stream;
    TP_LAUNCH(k_pm_green_table, pm_grid(half, kPmThreads), kPmThreads, 0, s, pm->green, n_mesh, r_cut, G);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        pm_release(pm);
        return TP_ERR_CUDA;
    }
    *out = pm;
    return TP_OK;
}

// The potential solve K in place: rho -> FFT -> x Green's function -> FFT^-1 -> rho.
static tp_status pm_solve(tp_pm *pm, cudaStream_t s)
{
    const int N = pm->N;
    const int64_t half = (int64_t)N * N * (N / 2 + 1);
    if (cufftSetStream(pm->fwd, s) != CUFFT_SUCCESS || cufftExecR2C(pm->fwd, pm->rho, pm->spec) != CUFFT_SUCCESS)
        return TP_ERR_CUDA;
    TP_LAUNCH(k_pm_green, pm_grid(half, kPmThreads), kPmThreads, 0, s, pm->spec, pm->green, half);
    if (cufftSetStream(pm->inv, s) != CUFFT_SUCCESS || cufftExecC2R(pm->inv, pm->spec, pm->rho) != CUFFT_SUCCESS)
        return TP_ERR_CUDA;
    return TP_OK;
}

// Steps 1-3 of the cycle: the mesh force of the current positions in amesh.
static tp_status pm_mesh_force(tp_pm *pm, const double *pos, const double *mass, int64_t n, cudaStream_t s)
{
    const int N = pm->N;
    const int64_t cells = (int64_t)N * N * N;
    cudaMemsetAsync(pm->rho, 0, sizeof(float) * cells, s);
    TP_LAUNCH(k_pm_assign, pm_grid(n, kPmThreads), kPmThreads, 0, s, pos, mass, n, N, (float)(1.0 / (double)n),
              pm->rho);
    const tp_status e = pm_solve(pm, s);
    if (e != TP_OK) return e;
    TP_LAUNCH(k_pm_gradient, pm_grid(cells, kPmThreads), kPmThreads, 0, s, pm->rho, pm->amesh, N);
    return TP_OK;
}

// The adjoint given the mesh force in amesh: U, div U, B = K div U, and the
// per-particle gradient.
static tp_status pm_adjoint(tp_pm *pm, const double *pos, const double *mass, int64_t n, const float *cot,
                            double *grad, int32_t accumulate, cudaStream_t s)
{
    const int N = pm->N;
    const int64_t cells = (int64_t)N * N * N;
    cudaMemsetAsync(pm->umesh, 0, sizeof(float4) * cells, s);
    TP_LAUNCH(k_pm_assign_vec, pm_grid(n, kPmThreads), kPmThreads, 0, s, pos, cot, n, N, pm->umesh);
    TP_LAUNCH(k_pm_divergence, pm_grid(cells, kPmThreads), kPmThreads, 0, s, pm->umesh, pm->rho, N);
    const tp_status e = pm_solve(pm, s);
    if (e != TP_OK) return e;
    TP_LAUNCH(k_pm_pack_w, pm_grid(cells, kPmThreads), kPmThreads, 0, s, pm->amesh, pm->rho, cells);
    TP_LAUNCH(k_pm_vjp_interp, pm_grid(n, kPmThreads), kPmThreads, 0, s, pos, mass, (float)(1.0 / (double)n), cot,
              n, N, pm->amesh, grad, accumulate);
    return TP_OK;
}

static tp_status pm_need_umesh(tp_pm *pm)
{
    if (pm->umesh) return TP_OK;
    const int64_t N = pm->N;
    if (cudaMalloc(&pm->umesh, sizeof(float4) * N * N * N) != cudaSuccess) {
        cudaGetLastError();
        pm->umesh = nullptr;
        return TP_ERR_OOM;
    }
    return TP_OK;
}

extern "C" tp_status tp_pm_force(tp_pm *pm, const double *pos, const double *mass, int64_t n, float *acc,
                                 int32_t accumulate, void *stream)
{
    NvtxRange range("PM");
    if (!pm || n < 0) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!is_dev(pos) || !is_dev(acc) || (mass && !is_dev(mass))) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const tp_status e = pm_mesh_force(pm, pos, mass, n, s);
    if (e != TP_OK) return e;
    TP_LAUNCH(k_pm_interp, pm_grid(n, kPmThreads), kPmThreads, 0, s, pos, n, pm->N, pm->amesh, acc, accumulate);
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

extern "C" tp_status tp_pm_vjp(tp_pm *pm, const double *pos, const double *mass, int64_t n, const float *cot,
                               double *grad, int32_t accumulate, void *stream)
{
    NvtxRange range("PM (adjoint)");
    if (!pm || n < 0) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!is_dev(pos) || !is_dev(cot) || !is_dev(grad) || (mass && !is_dev(mass))) return TP_ERR_INVALID_ARG;
    tp_status e = pm_need_umesh(pm);
    if (e != TP_OK) return e;
    cudaStream_t s = (cudaStream_t)stream;
    e = pm_mesh_force(pm, pos, mass, n, s);
    if (e == TP_OK) e = pm_adjoint(pm, pos, mass, n, cot, grad, accumulate, s);
    if (e != TP_OK) return e;
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

extern "C" tp_status tp_pm_force_vjp(tp_pm *pm, const double *pos, const double *mass, int64_t n, float *acc,
                                     const float *cot, double *grad, int32_t accumulate, void *stream)
{
    NvtxRange range("PM (forward and adjoint)");
    if (!pm || n < 0) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    if (!is_dev(pos) || !is_dev(acc) || !is_dev(cot) || !is_dev(grad) || (mass && !is_dev(mass)))
        return TP_ERR_INVALID_ARG;
    tp_status e = pm_need_umesh(pm);
    if (e != TP_OK) return e;
    cudaStream_t s = (cudaStream_t)stream;
    e = pm_mesh_force(pm, pos, mass, n, s);
    if (e != TP_OK) return e;
    TP_LAUNCH(k_pm_interp, pm_grid(n, kPmThreads), kPmThreads, 0, s, pos, n, pm->N, pm->amesh, acc, accumulate);
    e = pm_adjoint(pm, pos, mass, n, cot, grad, accumulate, s);
    if (e != TP_OK) return e;
    return cudaGetLastError() == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}

// which = 0: the potential of the last tp_pm_force call, [N^3]; which = 1:
// its -grad(phi) mesh, [N^3][3].  Synchronous.
extern "C" tp_status tp_pm_export_mesh(tp_pm *pm, int32_t which, float *host)
{
    if (!pm || !host || which < 0 || which > 1) return TP_ERR_INVALID_ARG;
    const int64_t N = pm->N, cells = N * N * N;
    cudaError_t e;
    if (which == 0) {
        e = cudaMemcpy(host, pm->rho, sizeof(float) * cells, cudaMemcpyDeviceToHost);
    } else {
        e = cudaMemcpy2D(host, 3 * sizeof(float), pm->amesh, sizeof(float4), 3 * sizeof(float), cells,
                         cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TP_ERR_CUDA;
    }
    return TP_OK;
}

extern "C" tp_status tp_pm_free(tp_pm *pm)
{
    if (pm) {
        cudaDeviceSynchronize();
        pm_release(pm);
    }
    return TP_OK;
}
