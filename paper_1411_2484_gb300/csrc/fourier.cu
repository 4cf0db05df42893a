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
// short transform runs radix-4 decimation-in-time stages (one radix-2 stage
// first when log2 of its length is odd) on bit-reversed input in shared
// memory.  FP64 throughout, as the paper's double-precision test; on GB300 the
// FP64 unit (2 fused multiply-adds per clock per SM) bounds these kernels.
#include <cuda_runtime.h>

#include "internal.h"

namespace phprng {

static constexpr int kFftThreads = 256;
static constexpr uint32_t kFftSmemBins = 2048;     // histograms this small go through shared memory
static constexpr uint32_t kColsElems = 2048;       // column block: C N1 complex values (32 KiB)

// Twiddle tables, one allocation: T[k] = w_M^k (k < M), then w_N1^t (t < N1),
// then w_N2^t (t < N2).
__global__ void __launch_bounds__(256) twiddle_kernel(double2 *__restrict__ tw, uint32_t M, uint32_t N1,
                                                      uint32_t N2)
{
    const uint32_t total = M + N1 + N2;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        uint32_t t = i, L = M;
        if (i >= M + N1) t = i - M - N1, L = N2;
        else if (i >= M) t = i - M, L = N1;
        double s, c;
        sincospi(2.0 * (double)t / (double)L, &s, &c);
        tw[i] = make_double2(c, s);
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }

// In-place transforms of nvec vectors of length L = 2^lg held in buf
// (bit-reversed order on entry, natural order on exit); tl[t] = w_L^t.
// A radix-4 step joins four consecutive length-h sub-transforms, which in the
// bit-reversed layout hold the samples of residues 0, 2, 1, 3 mod 4:
// X[pos + q h] = sum_r w_4h^(r pos) i^(r q) D_r[pos].
__device__ __forceinline__ void block_fft(double2 *buf, uint32_t lg, uint32_t nvec, const double2 *tl)
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
        const uint32_t q4 = L / 4, tstep = L / (4 * h);   // w_4h^x = tl[x tstep]
        for (uint32_t b = threadIdx.x; b < nvec * q4; b += blockDim.x) {
            const uint32_t v = b / q4, q = b % q4;
            const uint32_t pos = q & (h - 1);
            double2 *x = buf + v * L + (q - pos) * 4 + pos;
            double2 t0 = x[0], t2 = x[h], t1 = x[2 * h], t3 = x[3 * h];
            if (h > 1) {
                const uint32_t i1 = pos * tstep;
                t1 = cmul(t1, tl[i1]);
                t2 = cmul(t2, tl[2 * i1]);
                t3 = cmul(t3, tl[3 * i1]);
            }
            const double2 u0 = cadd(t0, t2), u1 = csub(t0, t2);
            const double2 u2 = cadd(t1, t3), u3 = mul_i(csub(t1, t3));
            x[0] = cadd(u0, u2);
            x[h] = cadd(u1, u3);
            x[2 * h] = csub(u0, u2);
            x[3 * h] = csub(u1, u3);
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
    const uint32_t M = 2 * N;
    block_fft(fbuf, lg1, C, tw + M);
    double2 *zo = Z + s * N;
    for (uint32_t e = threadIdx.x; e < C * N1; e += blockDim.x) {
        const uint32_t c = e % C, k1 = e / C, j2 = j20 + c;
        zo[(uint64_t)k1 * N2 + j2] = cmul(fbuf[c * N1 + k1], tw[2 * (j2 * k1)]);   // w_N^(j2 k1)
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

// X_k and, when both, X_(N-k) from a = Z_k and b = Z_(N-k).
__device__ __forceinline__ void emit(const FourierOut &o, const double2 *__restrict__ wM, uint32_t N, uint32_t k,
                                     double2 a, double2 b, bool both)
{
    const double2 bc = make_double2(b.x, -b.y);
    const double2 e2 = cadd(a, bc), d = csub(a, bc);
    const double2 o2 = make_double2(d.y, -d.x);               // 2 O_k = -i d
    const double2 p = cmul(wM[k], o2);
    const double2 xk = make_double2((e2.x + p.x) * o.scale, (e2.y + p.y) * o.scale);
    bin_part(o, xk.x);
    bin_part(o, xk.y);
    if (o.coef) o.coef[k] = xk;
    if (both) {
        const double2 xn = make_double2((e2.x - p.x) * o.scale, (p.y - e2.y) * o.scale);
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
    const uint32_t M = 2 * N;
    block_fft(fbuf, lg2, nvec, tw + M + N1);
    const double2 *A = fbuf, *B = fbuf + N2;
    if (j) {
        for (uint32_t t = threadIdx.x; t < N2; t += blockDim.x)
            emit(o, tw, N, rA + N1 * t, A[t], B[N2 - 1 - t], true);
    } else {
        const uint32_t h2 = N2 / 2;
        for (uint32_t t = threadIdx.x; t <= h2; t += blockDim.x)      // row 0: partner (N2 - t) mod N2
            emit(o, tw, N, N1 * t, A[t], A[(N2 - t) & (N2 - 1)], t != 0 && t != h2);
        if (nvec == 2)                                               // row N1/2: partner N2 - 1 - t
            for (uint32_t t = threadIdx.x; t < h2; t += blockDim.x)
                emit(o, tw, N, N1 / 2 + N1 * t, B[t], B[N2 - 1 - t], true);
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

int launch_twiddles(double2 *tw, uint32_t lgM, void *stream, std::string *err)
{
    uint32_t lgN, lg1;
    fourier_split(lgM, &lgN, &lg1);
    const uint32_t total = (uint32_t)fourier_twiddle_count(lgM);
    const uint32_t grid = (total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096;
    twiddle_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(tw, 1u << lgM, 1u << lg1, 1u << (lgN - lg1));
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
