// fourier.cu -- the Fourier test (Tests section): for sequences of M numbers,
// x_j = R_j - 1/2 and xhat_k = M^(-1/2) sum_j x_j exp(+2 pi i j k / M), k = 0 ..
// M/2 - 1; the real and imaginary parts of every xhat_k go to one histogram.
//
// The input is real, so one sequence is transformed as N = M/2 complex points
// z_j = x_2j + i x_(2j+1): with Z = DFT_N(z) (positive exponent),
//     E_k = (Z_k + conj Z_(N-k)) / 2,   O_k = (Z_k - conj Z_(N-k)) / 2i,
//     X_k = E_k + w_M^k O_k,   X_(N-k) = conj(E_k - w_M^k O_k)
// (w_L = exp(2 pi i / L); E and O are the transforms of the even and odd
// samples), which halves the FP64 work of a complex transform of M points.
//
// The N-point transform is the four-step decomposition N = N1 N2 (N1 <= 512,
// N2 <= 1024), j = N2 j1 + j2, k = k1 + N1 k2:
//     Z[k1 + N1 k2] = sum_j2 w_N2^(j2 k2) [ w_N^(j2 k1) sum_j1 z[N2 j1 + j2] w_N1^(j1 k1) ].
// fft_columns_kernel does the inner N1-point transforms (C adjacent columns j2
// per block, in shared memory) and the w_N^(j2 k1) factors into Z, row k1 of a
// sequence contiguous; fft_rows_kernel transforms rows k1 and N1 - k1 together
// (their outputs are the partners k, N - k above), forms X and bins it.  Each
// short transform runs radix-2 decimation-in-time stages two per pass (one
// single stage first when log2 of its length is odd) on bit-reversed input in shared
// memory, its butterflies in the six-multiply-add ratio form.  FP64 throughout,
// as the paper's double-precision test; on GB300 the FP64 unit (2 fused
// multiply-adds per clock per SM) bounds these kernels.
#include <cuda_runtime.h>

#include "internal.h"

namespace phprng {

static constexpr int kFftThreads = 256;
static constexpr uint32_t kFftSmemBins = 2048;     // histograms this small go through shared memory
static constexpr uint32_t kColsElems = 2048;       // column block: C N1 complex values (32 KiB)

// Twiddle tables, one allocation (N = M/2):
//   [0, N)            w_N^x = (cos, sin), the four-step factors;
//   [N, 2N)           w_M^k in ratio form scaled by 1/(2 sqrt M), the split;
//   [2N, 2N+N1)       w_N1^t in ratio form, the column transforms' factors;
//   [2N+N1, 2N+N1+N2) w_N2^t in ratio form, the row transforms' factors.
// Ratio form of w = c + i s at angle 2 pi t / L: outside the octants where
// |s| > |c| (ratio_quarter = 0) the pair (c, s/c), so w b = c (b + i (s/c) b);
// inside them (ratio_quarter = 1) w = s (1 + i r) i with r = -c/s, stored as
// (s, r), applied to i b.  The ratio's magnitude stays at most 1.
__device__ __forceinline__ uint32_t ratio_quarter(uint32_t t, uint32_t lgL)
{
    const uint32_t o = (uint32_t)(((uint64_t)t << 3) >> lgL);   // octant of 2 pi t / L
    return ((o + 1) >> 1) & 1u;
}

__global__ void __launch_bounds__(256) twiddle_kernel(double2 *__restrict__ tw, uint32_t lgM, uint32_t lg1,
                                                      uint32_t lg2, double scale)
{
    const uint32_t N = 1u << (lgM - 1), N1 = 1u << lg1, N2 = 1u << lg2;
    const uint32_t total = 2 * N + N1 + N2;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        uint32_t t, lg;
        double sc = 1.0;
        if (i < N) {
            double s, c;
            sincospi(2.0 * (double)i / (double)N, &s, &c);
            tw[i] = make_double2(c, s);
            continue;
        }
        if (i < 2 * N) t = i - N, lg = lgM, sc = scale;
        else if (i < 2 * N + N1) t = i - 2 * N, lg = lg1;
        else t = i - 2 * N - N1, lg = lg2;
        double s, c;
        sincospi(2.0 * (double)t / (double)(1u << lg), &s, &c);
        tw[i] = ratio_quarter(t, lg) ? make_double2(s * sc, -c / s) : make_double2(c * sc, s / c);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }

// i^q b by swapping and flipping sign bits (integer operations, no FP64 work).
__device__ __forceinline__ double2 rot_q(double2 b, uint32_t q)
{
    const bool odd = q & 1u;
    const long long x = __double_as_longlong(odd ? b.y : b.x), y = __double_as_longlong(odd ? b.x : b.y);
    const long long sx = (long long)((((q + 1) >> 1) & 1u)) << 63, sy = (long long)((q >> 1) & 1u) << 63;
    return make_double2(__longlong_as_double(x ^ sx), __longlong_as_double(y ^ sy));
}

// (a + w b, a - w b) with w in ratio form (m, r), b already turned by the
// quarter: six fused multiply-adds instead of four products and four sums.
__device__ __forceinline__ void bfly(double2 &o0, double2 &o1, double2 a, double2 b, double2 mr)
{
    const double u = fma(-mr.y, b.y, b.x), v = fma(mr.y, b.x, b.y);
    o0 = make_double2(fma(mr.x, u, a.x), fma(mr.x, v, a.y));
    o1 = make_double2(fma(-mr.x, u, a.x), fma(-mr.x, v, a.y));
}

// In-place transforms of nvec vectors of length L = 2^lg held in buf
// (bit-reversed order on entry, natural order on exit); rt[t] = w_L^t in
// ratio form.  Radix-2 decimation in time, its stages taken two at a time:
// one pass over a block of 4h joins the half-size-h pairs (pos, pos + h) and
// (pos + 2h, pos + 3h) by w_2h^pos, then the half-size-2h pairs (pos, pos + 2h)
// by w_4h^pos and (pos + h, pos + 3h) by w_4h^(pos + h) = i w_4h^pos; an odd
// log2 L starts with one plain radix-2 stage, and the first pass (h = 1, all
// factors 1 or i) is sums only.
__device__ __forceinline__ void block_fft(double2 *buf, uint32_t lg, uint32_t nvec, const double2 *rt)
{
    const uint32_t L = 1u << lg;
    uint32_t h = 1;
    if (lg & 1) {                                  // radix-2 first stage (all factors 1)
        for (uint32_t b = threadIdx.x; b < nvec * (L / 2); b += blockDim.x) {
            double2 *x = buf + 2 * b;
            const double2 a0 = x[0], a1 = x[1];
            x[0] = cadd(a0, a1);
            x[1] = csub(a0, a1);
        }
        __syncthreads();
        h = 2;
    }
    for (; h < L; h <<= 2) {
        const uint32_t q4 = L / 4, tstep = L / (4 * h);   // w_4h^x = rt[x tstep]
        for (uint32_t b = threadIdx.x; b < nvec * q4; b += blockDim.x) {
            const uint32_t v = b / q4, q = b % q4;
            const uint32_t pos = q & (h - 1);
            double2 *x = buf + v * L + (q - pos) * 4 + pos;
            const double2 x0 = x[0], x1 = x[h], x2 = x[2 * h], x3 = x[3 * h];
            double2 z0, z1, z2, z3;
            if (h == 1) {
                const double2 y0 = cadd(x0, x1), y1 = csub(x0, x1), y2 = cadd(x2, x3), y3 = mul_i(csub(x2, x3));
                z0 = cadd(y0, y2);
                z2 = csub(y0, y2);
                z1 = cadd(y1, y3);
                z3 = csub(y1, y3);
            } else {
                const uint32_t i2 = pos * tstep, i1 = 2 * i2;              // w_4h^pos, w_2h^pos
                const uint32_t q1 = ratio_quarter(i1, lg), q2 = ratio_quarter(i2, lg);
                const double2 w1 = rt[i1], w2 = rt[i2];
                double2 y0, y1, y2, y3;
                bfly(y0, y1, x0, rot_q(x1, q1), w1);
                bfly(y2, y3, x2, rot_q(x3, q1), w1);
                bfly(z0, z2, y0, rot_q(y2, q2), w2);
                bfly(z1, z3, y1, rot_q(y3, q2 + 1), w2);
            }
            x[0] = z0;
            x[h] = z1;
            x[2 * h] = z2;
            x[3 * h] = z3;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, uint32_t lg)
{
    return lg ? __brev(x) >> (32 - lg) : 0u;
}

// Block: sequence s, columns j20 .. j20 + C - 1.
__global__ void __launch_bounds__(kFftThreads)
fft_columns_kernel(const double2 *__restrict__ Rz, double2 *__restrict__ Z, uint32_t lgN, uint32_t lg1,
                   uint32_t C, const double2 *__restrict__ tw)
{
    extern __shared__ double2 fbuf[];
    const uint32_t N = 1u << lgN, N1 = 1u << lg1, N2 = N >> lg1, per_seq = N2 / C;
    const uint64_t s = blockIdx.x / per_seq;
    const uint32_t j20 = (blockIdx.x % per_seq) * C;
    const double2 *z = Rz + s * N;
    for (uint32_t e = threadIdx.x; e < C * N1; e += blockDim.x) {
        const uint32_t c = e % C, j1 = e / C;
        const double2 v = z[(uint64_t)N2 * j1 + j20 + c];
        fbuf[c * N1 + bitrev(j1, lg1)] = make_double2(v.x - 0.5, v.y - 0.5);
    }
    __syncthreads();
    block_fft(fbuf, lg1, C, tw + 2 * N);
    double2 *zo = Z + s * N;
    for (uint32_t e = threadIdx.x; e < C * N1; e += blockDim.x) {
        const uint32_t c = e % C, k1 = e / C, j2 = j20 + c;
        zo[(uint64_t)k1 * N2 + j2] = cmul(fbuf[c * N1 + k1], tw[j2 * k1]);   // w_N^(j2 k1)
    }
}

struct FourierOut {
    double scale;         // 1 / (2 sqrt(M))
    double w, inv;        // range [-w, w), nbins / 2w
    uint32_t nbins;
    unsigned int *sh;     // shared histogram or null
    unsigned long long *hist;
    double2 *coef;        // this sequence's M/2 coefficients or null
};

__device__ __forceinline__ void bin_part(const FourierOut &o, double v)
{
    int b = __double2int_rd((v + o.w) * o.inv);    // saturating conversion
    b = b < 0 ? 0 : (uint32_t)b > o.nbins - 1 ? (int)(o.nbins - 1) : b;
    if (o.sh) atomicAdd(o.sh + b, 1u);
    else atomicAdd(o.hist + b, 1ull);
}

// X_k and, when both, X_(N-k) from a = Z_k and b = Z_(N-k); wM[k] = w_M^k in
// ratio form with the scale 1/(2 sqrt M) folded into its multiplier.
__device__ __forceinline__ void emit(const FourierOut &o, const double2 *__restrict__ wM, uint32_t lgM,
                                     uint32_t N, uint32_t k, double2 a, double2 b, bool both)
{
    const double2 bc = make_double2(b.x, -b.y);
    const double2 e2 = cadd(a, bc), d = csub(a, bc);
    const double2 o2 = rot_q(d, 3 + ratio_quarter(k, lgM));   // 2 O_k = -i d, turned by the quarter
    const double2 mr = wM[k];
    const double u = fma(-mr.y, o2.y, o2.x), v = fma(mr.y, o2.x, o2.y);   // w O scaled = m (u, v)
    const double ex = e2.x * o.scale, ey = e2.y * o.scale;
    const double2 xk = make_double2(fma(mr.x, u, ex), fma(mr.x, v, ey));
    bin_part(o, xk.x);
    bin_part(o, xk.y);
    if (o.coef) o.coef[k] = xk;
    if (both) {
        const double2 xn = make_double2(fma(-mr.x, u, ex), fma(mr.x, v, -ey));
        bin_part(o, xn.x);
        bin_part(o, xn.y);
        if (o.coef) o.coef[N - k] = xn;
    }
}

// Block: sequence s, rows (j, N1 - j) for j >= 1; block 0 rows 0 and N1/2,
// each its own partner (row 0 alone when N1 = 1).
__global__ void __launch_bounds__(kFftThreads)
fft_rows_kernel(const double2 *__restrict__ Z, uint32_t lgN, uint32_t lg1, const double2 *__restrict__ tw,
                double scale, uint32_t nbins, double w, unsigned long long *__restrict__ hist,
                double2 *__restrict__ coef)
{
    extern __shared__ double2 fbuf[];
    const uint32_t N = 1u << lgN, N1 = 1u << lg1, lg2 = lgN - lg1, N2 = 1u << lg2;
    const uint32_t per_seq = N1 >= 2 ? N1 / 2 : 1, nvec = N1 >= 2 ? 2 : 1;
    const uint64_t s = blockIdx.x / per_seq;
    const uint32_t j = blockIdx.x % per_seq;
    const uint32_t rA = j, rB = j ? N1 - j : N1 / 2;
    FourierOut o;
    o.scale = scale;
    o.w = w;
    o.inv = (double)nbins / (2.0 * w);
    o.nbins = nbins;
    o.sh = nbins <= kFftSmemBins ? reinterpret_cast<unsigned int *>(fbuf + nvec * N2) : nullptr;
    o.hist = hist;
    o.coef = coef ? coef + s * N : nullptr;
    if (o.sh)
        for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x) o.sh[b] = 0;
    const double2 *zs = Z + s * N;
    for (uint32_t e = threadIdx.x; e < nvec * N2; e += blockDim.x) {
        const uint32_t v = e >> lg2, j2 = e & (N2 - 1);
        fbuf[v * N2 + bitrev(j2, lg2)] = zs[(uint64_t)(v ? rB : rA) * N2 + j2];
    }
    __syncthreads();
    block_fft(fbuf, lg2, nvec, tw + 2 * N + N1);
    const double2 *A = fbuf, *B = fbuf + N2, *wM = tw + N;
    const uint32_t lgM = lgN + 1;
    if (j) {
        for (uint32_t t = threadIdx.x; t < N2; t += blockDim.x)
            emit(o, wM, lgM, N, rA + N1 * t, A[t], B[N2 - 1 - t], true);
    } else {
        const uint32_t h2 = N2 / 2;
        for (uint32_t t = threadIdx.x; t <= h2; t += blockDim.x)      // row 0: partner (N2 - t) mod N2
            emit(o, wM, lgM, N, N1 * t, A[t], A[(N2 - t) & (N2 - 1)], t != 0 && t != h2);
        if (nvec == 2)                                               // row N1/2: partner N2 - 1 - t
            for (uint32_t t = threadIdx.x; t < h2; t += blockDim.x)
                emit(o, wM, lgM, N, N1 / 2 + N1 * t, B[t], B[N2 - 1 - t], true);
    }
    if (o.sh) {
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x)
            if (o.sh[b]) atomicAdd(hist + b, (unsigned long long)o.sh[b]);
    }
}

static void fourier_split(uint32_t lgM, uint32_t *lgN, uint32_t *lg1)
{
    *lgN = lgM - 1;
    *lg1 = *lgN / 2;
}

uint64_t fourier_twiddle_count(uint32_t lgM)
{
    uint32_t lgN, lg1;
    fourier_split(lgM, &lgN, &lg1);
    return (1ull << lgM) + (1ull << lg1) + (1ull << (lgN - lg1));
}

int launch_twiddles(double2 *tw, uint32_t lgM, double scale2, void *stream, std::string *err)
{
    uint32_t lgN, lg1;
    fourier_split(lgM, &lgN, &lg1);
    const uint32_t total = (uint32_t)fourier_twiddle_count(lgM);
    const uint32_t grid = (total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096;
    twiddle_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(tw, lgM, lg1, lgN - lg1, scale2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("twiddle_kernel launch: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

int launch_fourier(const double *R, uint64_t nseq, uint32_t lgM, const double2 *tw, double2 *Z,
                   uint32_t nbins, double w, double scale, uint64_t *hist, double *coef, void *stream,
                   std::string *err)
{
    if (nseq == 0) return PHPRNG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t lgN, lg1;
    fourier_split(lgM, &lgN, &lg1);
    const uint32_t N1 = 1u << lg1, N2 = 1u << (lgN - lg1);
    uint32_t C = kColsElems / N1;
    if (C > N2) C = N2;
    if (C > 16) C = 16;
    const uint64_t ga = nseq * (N2 / C), gb = nseq * (N1 >= 2 ? N1 / 2 : 1);
    fft_columns_kernel<<<(unsigned)ga, kFftThreads, C * N1 * sizeof(double2), s>>>(
        reinterpret_cast<const double2 *>(R), Z, lgN, lg1, C, tw);
    const uint32_t nvec = N1 >= 2 ? 2 : 1;
    const size_t smem_b = nvec * N2 * sizeof(double2) + (nbins <= kFftSmemBins ? nbins * 4 : 0);
    fft_rows_kernel<<<(unsigned)gb, kFftThreads, smem_b, s>>>(Z, lgN, lg1, tw, scale, nbins, w,
                                                               (unsigned long long *)hist, (double2 *)coef);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("Fourier kernels: ") + cudaGetErrorString(e);
        return PHPRNG_ECUDA;
    }
    return PHPRNG_OK;
}

}  // namespace phprng
