// Map kernels: magnification from counts (Eq. 12) and light curves of a
// Gaussian source along straight tracks (§4.1, Fig. 3).
#include "ml_internal.cuh"
#include "ml_alloc.h"

#include <algorithm>

#include <math.h>

#include <mutex>

namespace ml {

// mu_ij = N_ij * S_I / S_S (Eq. 12).  Vectorised: four pixels per thread per step,
// uint4 loads and float4 / double2 stores, grid-stride over the map.
__global__ void k_mu_u32_f32(const uint4 *__restrict__ in, float4 *__restrict__ out, int64_t n4,
                             float scale)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 v = __ldcs(in + i);
        __stcs(out + i, make_float4((float)v.x * scale, (float)v.y * scale, (float)v.z * scale,
                                    (float)v.w * scale));
    }
}

__global__ void k_mu_u32_f64(const uint4 *__restrict__ in, double2 *__restrict__ out, int64_t n4,
                             double scale)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 v = __ldcs(in + i);
        __stcs(out + 2 * i, make_double2((double)v.x * scale, (double)v.y * scale));
        __stcs(out + 2 * i + 1, make_double2((double)v.z * scale, (double)v.w * scale));
    }
}

__global__ void k_mu_f32(const float4 *__restrict__ in, float4 *__restrict__ out, int64_t n4,
                         float scale)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = __ldcs(in + i);
        __stcs(out + i, make_float4(v.x * scale, v.y * scale, v.z * scale, v.w * scale));
    }
}

__global__ void k_mu_f32_f64(const float4 *__restrict__ in, double2 *__restrict__ out, int64_t n4,
                             double scale)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = __ldcs(in + i);
        __stcs(out + 2 * i, make_double2((double)v.x * scale, (double)v.y * scale));
        __stcs(out + 2 * i + 1, make_double2((double)v.z * scale, (double)v.w * scale));
    }
}

// Scalar tail (maps whose pixel count is not a multiple of 4).
__global__ void k_mu_tail(const uint32_t *cu, const float *cf, int want, void *out, int64_t from,
                          int64_t n, double scale)
{
    int64_t i = from + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = cu ? (double)cu[i] : (double)cf[i];
    if (want == ML_MAP_MU_F32) reinterpret_cast<float *>(out)[i] = (float)(v * scale);
    else reinterpret_cast<double *>(out)[i] = v * scale;
}

cudaError_t launch_mu(const Geo &g, const uint32_t *cu, const float *cf, int want, void *out,
                      double scale, cudaStream_t s)
{
    int64_t n = (int64_t)g.mnx * g.mny, n4 = n / 4;
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (n4 > 0) {
        if (cu && want == ML_MAP_MU_F32)
            k_mu_u32_f32<<<(unsigned)blocks, 256, 0, s>>>((const uint4 *)cu, (float4 *)out, n4,
                                                          (float)scale);
        else if (cu)
            k_mu_u32_f64<<<(unsigned)blocks, 256, 0, s>>>((const uint4 *)cu, (double2 *)out, n4,
                                                          scale);
        else if (want == ML_MAP_MU_F32)
            k_mu_f32<<<(unsigned)blocks, 256, 0, s>>>((const float4 *)cf, (float4 *)out, n4,
                                                      (float)scale);
        else
            k_mu_f32_f64<<<(unsigned)blocks, 256, 0, s>>>((const float4 *)cf, (double2 *)out, n4,
                                                          scale);
    }
    if (n > 4 * n4)
        k_mu_tail<<<1, 32, 0, s>>>(cu, cf, want, out, 4 * n4, n, scale);
    return cudaGetLastError();
}

// Light curves (§4.1, Fig. 3).  For every sample: bilinear interpolation between the four
// pixel centres around the point, each value being the map convolved with
// the separable normalised Gaussian taps (zero outside the map).  Only the
// pixels the samples need are convolved.  One warp per sample group; taps
// in shared memory.
__global__ void k_light_curves(Geo g, const uint32_t *__restrict__ cu, const float *__restrict__ cf,
                               double scale, const double *__restrict__ tracks, int n_tracks,
                               int n_samples, int h, const float *__restrict__ taps_g,
                               float *__restrict__ out)
{
    __shared__ float taps[129];
    for (int t = threadIdx.x; t <= 2 * h; t += blockDim.x) taps[t] = taps_g[t];
    __syncthreads();
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_tracks * n_samples) return;
    int tr = (int)(q / n_samples), k = (int)(q % n_samples);
    const double *T = tracks + 4 * tr;
    double t = n_samples > 1 ? (double)k / (double)(n_samples - 1) : 0.0;
    double u = T[0] + t * (T[2] - T[0]) - 0.5;
    double v = T[1] + t * (T[3] - T[1]) - 0.5;
    double fu = floor(u), fv = floor(v);
    double wx = u - fu, wy = v - fv;
    int i0 = (int)fu, j0 = (int)fv;
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) {
        int pi = i0 + (c & 1), pj = j0 + (c >> 1);
        double wc = ((c & 1) ? wx : 1.0 - wx) * ((c >> 1) ? wy : 1.0 - wy);
        if (pi < 0 || pi >= g.mnx || pj < 0 || pj >= g.mny || wc == 0.0) continue;
        double conv = 0.0;
        for (int dy = -h; dy <= h; ++dy) {
            int yy = pj + dy;
            if (yy < 0 || yy >= g.mny) continue;
            double row = 0.0;
            const int64_t base = (int64_t)yy * g.mnx;
            for (int dx = -h; dx <= h; ++dx) {
                int xx = pi + dx;
                if (xx < 0 || xx >= g.mnx) continue;
                double val = cu ? (double)cu[base + xx] : (double)cf[base + xx];
                row += (double)taps[dx + h] * val;
            }
            conv += (double)taps[dy + h] * row;
        }
        acc += wc * conv;
    }
    out[q] = (float)(acc * scale);
}

// Normalised Gaussian source taps of §4.1 at integer offsets |t| <= floor(4 sigma),
// truncated there and scaled to sum 1; one function for every light-curve path
// so that they agree bit for bit.  Returns the half-width h, or -1 above 64.
int light_curve_taps(double sigma_px, float taps[129])
{
    int h = (int)floor(4.0 * sigma_px);
    if (h > 64) return -1;
    double sum = 0.0, w[129];
    for (int t = -h; t <= h; ++t) {
        w[t + h] = exp(-0.5 * ((double)t / sigma_px) * ((double)t / sigma_px));
        sum += w[t + h];
    }
    for (int t = 0; t <= 2 * h; ++t) taps[t] = (float)(w[t] / sum);
    return h;
}

// ---- light curves without allocation -----------------------------------------
//
// Scratch for the allocation-free light-curve entry point: the Gaussian taps
// (first 1024 bytes) and the device copy of the tracks (32 bytes each).  It is
// a fixed array in the library's device image, present on every device that
// loads the library until the process exits.  Every call overwrites what it
// uses, so nothing in it has to start at zero; calls share it, so two calls
// that overlap on the GPU race (order them on one stream).
constexpr size_t LC_TAPS_BYTES = 1024;
static __device__ __align__(256) unsigned char g_lc_scratch[LC_TAPS_BYTES + 32 * ML_NOALLOC_MAX_TRACKS];

// Device address of g_lc_scratch, looked up once per device (with that device
// current): in host code the array's name is only a host-side stand-in.
static cudaError_t lc_scratch_address(unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[1024] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 1024) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

cudaError_t launch_light_curves_noalloc(const Geo &g, const uint32_t *cu, const float *cf,
                                        double scale, const double *tracks_host, int n_tracks,
                                        int n_samples, double sigma_px, float *out, cudaStream_t s)
{
    float taps[129];
    int h = light_curve_taps(sigma_px, taps);
    if (h < 0 || n_tracks > ML_NOALLOC_MAX_TRACKS) return cudaErrorInvalidValue;
    unsigned char *base = nullptr;
    cudaError_t e = lc_scratch_address(&base);
    if (e != cudaSuccess) return e;
    float *d_taps = reinterpret_cast<float *>(base);
    double *d_tracks = reinterpret_cast<double *>(base + LC_TAPS_BYTES);
    e = cudaMemcpyAsync(d_taps, taps, sizeof(float) * (2 * h + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_tracks, tracks_host, sizeof(double) * 4 * (size_t)n_tracks,
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    int64_t n = (int64_t)n_tracks * n_samples;
    k_light_curves<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, cu, cf, scale, d_tracks, n_tracks,
                                                               n_samples, h, d_taps, out);
    return cudaGetLastError();
}

cudaError_t launch_light_curves(const Geo &g, const uint32_t *cu, const float *cf, double scale,
                                const double *tracks, int n_tracks, int n_samples,
                                double sigma_px, float *out, cudaStream_t s)
{
    float taps[129];
    int h = light_curve_taps(sigma_px, taps);
    if (h < 0) return cudaErrorInvalidValue;
    float *d_taps = nullptr;
    cudaError_t e = ml_malloc_async((void **)&d_taps, sizeof(float) * (2 * h + 1), s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_taps, taps, sizeof(float) * (2 * h + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { cudaFreeAsync(d_taps, s); return e; }
    int64_t n = (int64_t)n_tracks * n_samples;
    k_light_curves<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, cu, cf, scale, tracks, n_tracks,
                                                               n_samples, h, d_taps, out);
    e = cudaGetLastError();
    cudaFreeAsync(d_taps, s);
    return e;
}

// Light curves with the taps and tracks already on the device (the batched
// step, which is captured in a CUDA graph and must not allocate).
cudaError_t launch_light_curves_dev(const Geo &g, const uint32_t *cu, const float *cf, double scale,
                                    const double *d_tracks, int n_tracks, int n_samples, int h,
                                    const float *d_taps, float *out, cudaStream_t s)
{
    int64_t n = (int64_t)n_tracks * n_samples;
    if (n == 0) return cudaSuccess;
    k_light_curves<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, cu, cf, scale, d_tracks, n_tracks,
                                                               n_samples, h, d_taps, out);
    return cudaGetLastError();
}

// ---- 64-bit sum of a count map -------------------------------------------------
//
// The shooting kernels add counts with fire-and-forget atomics, so a wrapped
// uint32 pixel is not seen there; it shows as a map sum (taken in 64 bits)
// that falls short of the in-map ray counter by a multiple of 2^32.
__global__ void k_map_sum(const uint32_t *__restrict__ map, size_t n, unsigned long long *sum)
{
    unsigned long long acc = 0;
    const size_t n4 = n / 4;
    const uint4 *m4 = reinterpret_cast<const uint4 *>(map);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = m4[i];
        acc += (unsigned long long)v.x + v.y + (unsigned long long)v.z + v.w;
    }
    for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        acc += map[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

cudaError_t launch_map_sum(const uint32_t *map, size_t n, unsigned long long *sum, int num_sms,
                           cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const size_t want = (n / 4 + 255) / 256;
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)num_sms * 8));
    k_map_sum<<<blocks, 256, 0, s>>>(map, n, sum);
    return cudaGetLastError();
}

// ---- peak identification on light curves (§4.2) ---------------------------------
//
// Curves run along x (a map row is a curve; its neighbours are the rows above
// and below) or along y.  Candidate at position j of curve i: N > both
// neighbours along the curve and (2N - a - b)^2 > 3 k^2 (a + N + b), the
// squared form of N - <N> > k sqrt(<N>), compared in FP64 (exact for counts
// below 2^26).  True peak: a candidate with a candidate among positions
// j-1..j+1 of both neighbouring curves.
__device__ __forceinline__ uint32_t peak_count(const uint32_t *N, int nx, int c, int j, int along)
{
    return along == 0 ? N[(size_t)c * nx + j] : N[(size_t)j * nx + c];
}

__global__ void k_peak_candidates(const uint32_t *__restrict__ N, int nx, int ny, int along,
                                  double k2x3, uint8_t *__restrict__ mask)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)nx * ny) return;
    const int ix = (int)(q % nx), iy = (int)(q / nx);
    const int len = along == 0 ? nx : ny;          // positions along a curve
    const int j = along == 0 ? ix : iy, c = along == 0 ? iy : ix;
    uint8_t m = 0;
    if (j > 0 && j < len - 1) {
        const uint32_t a = peak_count(N, nx, c, j - 1, along), v = peak_count(N, nx, c, j, along),
                       b = peak_count(N, nx, c, j + 1, along);
        if (v > a && v > b) {
            const double d = 2.0 * (double)v - (double)a - (double)b;
            if (d * d > k2x3 * ((double)a + (double)v + (double)b)) m = 1;
        }
    }
    mask[q] = m;
}

__global__ void k_peak_validate(int nx, int ny, int along, uint8_t *__restrict__ mask,
                                int32_t *__restrict__ peaks, int64_t capacity,
                                unsigned long long *__restrict__ found)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)nx * ny) return;
    if (!(mask[q] & 1)) return;
    const int ix = (int)(q % nx), iy = (int)(q / nx);
    const int ncurves = along == 0 ? ny : nx, len = along == 0 ? nx : ny;
    const int j = along == 0 ? ix : iy, c = along == 0 ? iy : ix;
    if (c == 0 || c == ncurves - 1) return;
    bool lo = false, hi = false;
    for (int dj = -1; dj <= 1; ++dj) {
        const int jj = j + dj;
        if (jj < 0 || jj >= len) continue;
        const size_t ql = along == 0 ? (size_t)(c - 1) * nx + jj : (size_t)jj * nx + (c - 1);
        const size_t qh = along == 0 ? (size_t)(c + 1) * nx + jj : (size_t)jj * nx + (c + 1);
        lo |= (mask[ql] & 1) != 0;
        hi |= (mask[qh] & 1) != 0;
    }
    if (!(lo && hi)) return;
    // bit 1 only: other threads read bit 0 of this byte concurrently
    atomicOr(reinterpret_cast<unsigned int *>(mask + (q & ~(int64_t)3)), 2u << (8 * (q & 3)));
    const unsigned long long slot = atomicAdd(found, 1ull);
    if ((int64_t)slot < capacity) {
        peaks[2 * slot] = ix;
        peaks[2 * slot + 1] = iy;
    }
}

cudaError_t launch_peaks(const uint32_t *N, int nx, int ny, int along, double nsigma, uint8_t *mask,
                         int32_t *peaks, int64_t capacity, unsigned long long *found, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny;
    cudaError_t e = cudaMemsetAsync(found, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_peak_candidates<<<blocks, 256, 0, s>>>(N, nx, ny, along, 3.0 * nsigma * nsigma, mask);
    k_peak_validate<<<blocks, 256, 0, s>>>(nx, ny, along, mask, peaks, capacity, found);
    return cudaGetLastError();
}

// ---- peak statistics over distance to the caustic (§4.2, Figs. 4-5) ------------
//
// Position j along a curve has the distance d = |origin + (j + 1/2) step - caustic|
// of its pixel centre, formed with separately rounded FP64 operations (no fused
// multiply-add), so that the bin it falls in does not depend on the compiler;
// bin b holds edges[b] <= d < edges[b+1].  The curves' end positions hold no
// peak and fall in no bin.
__global__ void k_peak_bins(int len, double origin, double step, double caustic,
                            const double *__restrict__ edges, int nbins,
                            unsigned long long per_position, int32_t *__restrict__ bin_of,
                            unsigned long long *__restrict__ n_positions)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    int b = -1;
    if (j > 0 && j < len - 1) {
        const double c = __dadd_rn(origin, __dmul_rn((double)j + 0.5, step));
        const double d = fabs(__dadd_rn(c, -caustic));
        if (d >= edges[0] && d < edges[nbins]) {
            int lo = 0, hi = nbins;                 // edges[lo] <= d < edges[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (edges[mid] <= d) lo = mid; else hi = mid;
            }
            b = lo;
        }
    }
    bin_of[j] = b;
    if (b >= 0 && per_position) atomicAdd(&n_positions[b], per_position);
}

// Per bin: the true peaks (mask bit 1) and the sum of their counts, gathered in
// shared memory (2 nbins 64-bit counters) and added to the global sums once per
// block.  Integer sums: the result does not depend on the order.
__global__ void k_peak_stats(const uint8_t *__restrict__ mask, const uint32_t *__restrict__ N, int nx,
                             int ny, int along, const int32_t *__restrict__ bin_of, int nbins,
                             unsigned long long *__restrict__ n_peaks,
                             unsigned long long *__restrict__ sum_counts)
{
    extern __shared__ unsigned long long sh_bins[];
    for (int b = threadIdx.x; b < 2 * nbins; b += blockDim.x) sh_bins[b] = 0;
    __syncthreads();
    const int64_t n = (int64_t)nx * ny;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (!(mask[q] & 2)) continue;
        const int j = along == 0 ? (int)(q % nx) : (int)(q / nx);
        const int b = bin_of[j];
        if (b < 0) continue;
        atomicAdd(&sh_bins[b], 1ull);
        atomicAdd(&sh_bins[nbins + b], (unsigned long long)N[q]);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (sh_bins[b] == 0) continue;
        atomicAdd(&n_peaks[b], sh_bins[b]);
        atomicAdd(&sum_counts[b], sh_bins[nbins + b]);
    }
}

cudaError_t launch_peak_stats(const uint32_t *N, int nx, int ny, int along, const uint8_t *mask,
                              double origin, double step, double caustic, const double *edges,
                              int nbins, int32_t *bin_of, unsigned long long *out, int num_sms,
                              cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 3 * (size_t)nbins * sizeof(unsigned long long), s);
    const int len = along == 0 ? nx : ny, ncurves = along == 0 ? ny : nx;
    if (e != cudaSuccess || len == 0 || ncurves == 0) return e;
    const unsigned long long per_position = ncurves >= 3 ? (unsigned long long)(ncurves - 2) : 0ull;
    k_peak_bins<<<(len + 255) / 256, 256, 0, s>>>(len, origin, step, caustic, edges, nbins, per_position,
                                                  bin_of, out + 2 * (size_t)nbins);
    const int64_t n = (int64_t)nx * ny;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
    k_peak_stats<<<blocks, 256, 2 * (size_t)nbins * sizeof(unsigned long long), s>>>(
        mask, N, nx, ny, along, bin_of, nbins, out, out + nbins);
    return cudaGetLastError();
}

// ---- adjoint of the light curves ---------------------------------------------
//
// A light-curve sample is L = sum_c w_c sum_{dx,dy} taps[dx] taps[dy] M[p_c + (dx, dy)]
// over the four bilinear corners p_c (k_light_curves), a linear map of the
// magnification map M.  Its transpose adds, for every sample with incoming
// gradient g, g w_c taps[dx] taps[dy] to the same pixels, skipping exactly the
// corners and taps the forward skips.
__global__ void k_light_curves_adj(int mnx, int mny, const double *__restrict__ tracks, int n_tracks,
                                   int n_samples, int h, const float *__restrict__ taps_g,
                                   const float *__restrict__ dl, float *__restrict__ gmap)
{
    __shared__ float taps[129];
    for (int t = threadIdx.x; t <= 2 * h; t += blockDim.x) taps[t] = taps_g[t];
    __syncthreads();
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)n_tracks * n_samples) return;
    const float gq = dl[q];
    if (gq == 0.f) return;
    int tr = (int)(q / n_samples), k = (int)(q % n_samples);
    const double *T = tracks + 4 * tr;
    double t = n_samples > 1 ? (double)k / (double)(n_samples - 1) : 0.0;
    double u = T[0] + t * (T[2] - T[0]) - 0.5;
    double v = T[1] + t * (T[3] - T[1]) - 0.5;
    double fu = floor(u), fv = floor(v);
    double wx = u - fu, wy = v - fv;
    int i0 = (int)fu, j0 = (int)fv;
    for (int c = 0; c < 4; ++c) {
        int pi = i0 + (c & 1), pj = j0 + (c >> 1);
        double wc = ((c & 1) ? wx : 1.0 - wx) * ((c >> 1) ? wy : 1.0 - wy);
        if (pi < 0 || pi >= mnx || pj < 0 || pj >= mny || wc == 0.0) continue;
        const float gw = (float)((double)gq * wc);
        for (int dy = -h; dy <= h; ++dy) {
            int yy = pj + dy;
            if (yy < 0 || yy >= mny) continue;
            const float gy = gw * taps[dy + h];
            for (int dx = -h; dx <= h; ++dx) {
                int xx = pi + dx;
                if (xx < 0 || xx >= mnx) continue;
                atomicAdd(gmap + (int64_t)yy * mnx + xx, gy * taps[dx + h]);
            }
        }
    }
}

cudaError_t launch_light_curves_adj(int mnx, int mny, const double *d_tracks, int n_tracks,
                                    int n_samples, double sigma_px, const float *dl, float *gmap,
                                    cudaStream_t s)
{
    float taps[129];
    const int h = light_curve_taps(sigma_px, taps);
    if (h < 0) return cudaErrorInvalidValue;
    float *d_taps = nullptr;
    cudaError_t e = ml_malloc_async((void **)&d_taps, sizeof(float) * (2 * h + 1), s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_taps, taps, sizeof(float) * (2 * h + 1), cudaMemcpyHostToDevice, s);
    const int64_t n = (int64_t)n_tracks * n_samples;
    if (e == cudaSuccess && n > 0) {
        k_light_curves_adj<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(mnx, mny, d_tracks, n_tracks,
                                                                        n_samples, h, d_taps, dl, gmap);
        e = cudaGetLastError();
    }
    cudaFreeAsync(d_taps, s);
    return e;
}

}  // namespace ml
