// circ.cu -- products with a circulant multiplier through the DFT
// (Thm. 2.1: a Toeplitz, hence circulant, matrix times a vector costs
// O(n log n); here every row of A is such a product).
//
// For a real first column g, G[i][j] = g[(i-j) mod n]:
//   (v G)_j   = sum_i v_i g_{i-j}   -> DFT: v^ * conj(g^)   (mode 0, C = A G row by row)
//   (G v)_i   = sum_j g_{i-j} v_j   -> DFT: g^ * v^         (mode 1, x = G y)
//   (G^T v)_i = sum_j g_{j-i} v_j   -> DFT: v^ * conj(g^)   (mode 2, adjoint)
// Two real vectors are packed as the real and imaginary parts of one complex
// vector; because g^ is the transform of a real sequence both results come
// back real, in the real and imaginary parts.  One CTA per pair of vectors:
// the whole length-n complex vector sits in shared memory (n <= 8192 in FP64),
// a radix-2 decimation-in-frequency pass leaves the spectrum in bit-reversed
// order, the product with the (bit-reversed, 1/n-scaled) spectrum of g is
// taken in that order, and a decimation-in-time pass with conjugate
// twiddles returns the natural order, so no permutation is ever done.
// A Toeplitz multiplier of order n is the leading n x n block of a circulant
// of order cn = 2n (first column t_0 .. t_{n-1}, 0, t_{-(n-1)} .. t_{-1}):
// its products read n entries per vector, zero the rest, and keep the first
// n results.
#include "genp_internal.cuh"

#include <math.h>

#include <type_traits>

namespace genp {
namespace {

constexpr int kThreads = 512;
constexpr int kMaxLogN = 13;  // 8192 complex doubles = 128 KiB of shared memory

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
    C2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename R, typename C2>
__device__ void dif_forward(C2 *z, const C2 *tw, int logn) {
    const int n = 1 << logn;
    for (int lh = logn - 1, ts = 1; lh >= 0; --lh, ts <<= 1) {
        const int h = 1 << lh;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int j = b & (h - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + j, i1 = i0 + h;
            const C2 a = z[i0], c = z[i1];
            C2 s, d;
            s.x = a.x + c.x; s.y = a.y + c.y;
            d.x = a.x - c.x; d.y = a.y - c.y;
            z[i0] = s;
            z[i1] = cmul(d, tw[j * ts]);
        }
        __syncthreads();
    }
}

template <typename R, typename C2>
__device__ void dit_inverse(C2 *z, const C2 *tw, int logn) {
    const int n = 1 << logn;
    for (int lh = 0, ts = n >> 1; lh < logn; ++lh, ts >>= 1) {
        const int h = 1 << lh;
        for (int b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
            const int j = b & (h - 1);
            const int i0 = ((b >> lh) << (lh + 1)) + j, i1 = i0 + h;
            C2 w = tw[j * ts];
            w.y = -w.y;
            const C2 a = z[i0], c = cmul(z[i1], w);
            C2 s, d;
            s.x = a.x + c.x; s.y = a.y + c.y;
            d.x = a.x - c.x; d.y = a.y - c.y;
            z[i0] = s;
            z[i1] = d;
        }
        __syncthreads();
    }
}

__global__ void k_twiddles(double2 *tw, float2 *tw32, int logn) {
    const int n = 1 << logn;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < (n >> 1); k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)k / (double)n, &s, &c);
        tw[k] = make_double2(c, -s);
        tw32[k] = make_float2((float)c, (float)(-s));
    }
}

// spec = DFT(g)/n in bit-reversed order (FP64 and an FP32 copy).
__global__ void k_spectrum(const double *g, const double2 *tw, int logn, double2 *spec, float2 *spec32) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double2 *z = reinterpret_cast<double2 *>(smraw);
    const int n = 1 << logn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = make_double2(g[i], 0.0);
    __syncthreads();
    dif_forward<double>(z, tw, logn);
    const double inv = 1.0 / (double)n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double2 v = make_double2(z[k].x * inv, z[k].y * inv);
        spec[k] = v;
        spec32[k] = make_float2((float)v.x, (float)v.y);
    }
}

template <typename TI, typename TO, typename R>
__global__ void __launch_bounds__(kThreads)
k_circ_apply(const typename Cx<R>::T *spec, const typename Cx<R>::T *tw, int logn, int mode, const TI *in,
             int64_t ips, int64_t ies, TO *out, int64_t ops, int64_t oes, int64_t count, int accumulate,
             int nin, int nout, const int *skip) {
    using C2 = typename Cx<R>::T;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    C2 *z = reinterpret_cast<C2 *>(smraw);
    const int n = 1 << logn;
    const int64_t p0 = 2 * (int64_t)blockIdx.x;
    const bool two = p0 + 1 < count;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {   // zero past nin (Toeplitz embedding)
        C2 v;
        v.x = i < nin ? (R)in[p0 * ips + i * ies] : R(0);
        v.y = (two && i < nin) ? (R)in[(p0 + 1) * ips + i * ies] : R(0);
        z[i] = v;
    }
    __syncthreads();
    dif_forward<R>(z, tw, logn);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        C2 h = spec[k];
        if (mode != 1) h.y = -h.y;
        z[k] = cmul(z[k], h);
    }
    __syncthreads();
    dit_inverse<R>(z, tw, logn);
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
        const C2 v = z[i];
        TO *o0 = out + p0 * ops + i * oes;
        *o0 = accumulate ? (TO)((R)*o0 + v.x) : (TO)v.x;
        if (two) {
            TO *o1 = out + (p0 + 1) * ops + i * oes;
            *o1 = accumulate ? (TO)((R)*o1 + v.y) : (TO)v.y;
        }
    }
}

int ilog2(int64_t n) {
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

}  // namespace

bool circ_fft_supported(int64_t n) { return n >= 2 && n <= (1 << kMaxLogN) && (n & (n - 1)) == 0; }

cudaError_t circ_prepare(genp_multiplier *G, cudaStream_t s) {
    if (!circ_fft_supported(G->cn)) return cudaSuccess;
    const int logn = ilog2(G->cn);
    const size_t sm = (size_t)G->cn * sizeof(double2);
    cudaFuncSetAttribute(k_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    note_launch();
    k_twiddles<<<(unsigned)cdiv(G->cn / 2, 256), 256, 0, s>>>(G->twid, G->twid_f32, logn);
    note_launch();
    k_spectrum<<<1, kThreads, sm, s>>>(G->g, G->twid, logn, G->spec, G->spec_f32);
    return cudaGetLastError();
}

namespace {
template <typename TI, typename TO, typename R>
cudaError_t circ_apply_impl(const genp_multiplier *G, int mode, const TI *in, int64_t ips, int64_t ies, TO *out,
                            int64_t ops, int64_t oes, int64_t count, int accumulate, const int *skip,
                            cudaStream_t s) {
    using C2 = typename Cx<R>::T;
    if (!circ_fft_supported(G->cn)) return cudaErrorInvalidValue;
    if (count <= 0) return cudaSuccess;
    const int logn = ilog2(G->cn);
    const size_t sm = (size_t)G->cn * sizeof(C2);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_circ_apply<TI, TO, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t(1) << kMaxLogN) * sizeof(C2)));
        attr = true;
    }
    const C2 *spec = sizeof(R) == 8 ? (const C2 *)G->spec : (const C2 *)G->spec_f32;
    const C2 *tw = sizeof(R) == 8 ? (const C2 *)G->twid : (const C2 *)G->twid_f32;
    const int64_t blocks = cdiv(count, 2);
    if (blocks > 2147483647) return cudaErrorInvalidValue;
    note_launch();
    k_circ_apply<TI, TO, R><<<(unsigned)blocks, kThreads, sm, s>>>(spec, tw, logn, mode, in, ips, ies, out, ops, oes,
                                                                    count, accumulate, (int)G->n, (int)G->n, skip);
    return cudaGetLastError();
}
}  // namespace

template <typename TI, typename TO>
cudaError_t circ_apply(const genp_multiplier *G, int mode, const TI *in, int64_t ips, int64_t ies, TO *out,
                       int64_t ops, int64_t oes, int64_t count, const int *skip, cudaStream_t s) {
    using R = typename std::conditional<sizeof(TO) == 8, double, float>::type;
    return circ_apply_impl<TI, TO, R>(G, mode, in, ips, ies, out, ops, oes, count, 0, skip, s);
}
template cudaError_t circ_apply<double, double>(const genp_multiplier *, int, const double *, int64_t, int64_t,
                                                double *, int64_t, int64_t, int64_t, const int *, cudaStream_t);
template cudaError_t circ_apply<float, float>(const genp_multiplier *, int, const float *, int64_t, int64_t, float *,
                                              int64_t, int64_t, int64_t, const int *, cudaStream_t);
template cudaError_t circ_apply<double, float>(const genp_multiplier *, int, const double *, int64_t, int64_t, float *,
                                               int64_t, int64_t, int64_t, const int *, cudaStream_t);

// X (+)= G Y or G^T Y on the columns of Y (n x nrhs, double).
cudaError_t circ_apply_cols(const genp_multiplier *G, bool trans, const double *Y, int64_t ldy, double *X, int64_t ldx,
                            int64_t nrhs, bool accumulate, const int *skip, cudaStream_t s) {
    return circ_apply_impl<double, double, double>(G, trans ? 2 : 1, Y, 1, ldy, X, 1, ldx, nrhs, accumulate ? 1 : 0,
                                                   skip, s);
}

}  // namespace genp
