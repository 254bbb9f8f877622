/*
 * optigpu_oracle.c -- the plain, slow CPU oracle for the transpose and the
 * sum reduction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no header, helper, constant or table with the
 * CUDA path: the element decoders below are written here from the IEEE-754
 * binary16 and bfloat16 format definitions, not taken from any CUDA header.
 *
 * What it computes (thesis "Source-to-Source Transformations for GPU Code
 * Generation", arxiv 2605.13864):
 *
 *   transpose  Listing 3.5, Sec. 3.1: out[x][y] = in[y][x] for x < W, y < H.
 *              With rows = H and cols = W and both matrices dense row-major
 *              (the generated kernel of Listing 6.21, Sec. 6, indexes the
 *              input as MINDEX2(H, W, ...) and the output as MINDEX2(W, H,
 *              ...)), this is dst[c * rows + r] = src[r * cols + c].  The
 *              copy is a byte copy of one element, so every bit pattern
 *              (NaN payloads, -0) survives.
 *
 *   reduce     Listing 2.1, Sec. 2.1: the result is reduce_sum(N, A), the sum
 *              of A(0) .. A(N-1), computed by a sequential loop.  Integer
 *              input is summed exactly in int64.  Float input (fp32, bf16,
 *              fp16) is widened exactly to double and summed sequentially in
 *              double; a Neumaier-compensated double sum and the double sum of
 *              absolute values are offered beside it for error reporting.
 *
 *   tiled forms  Listing 3.8, Sec. 3.2 (the 32x32 tile loop nest of the
 *              transpose) and Listing 2.2, Sec. 2.2.1 (the partial-sum form
 *              of the reduction: per-chunk sums, then a sequential sum of the
 *              chunk sums).  The listings assume the sizes divide the tile;
 *              here the last tile or chunk is simply shorter.
 *
 * Parity pins (see tests/test_oracle.py): closed forms (sum of 0..n-1, the
 * index-matrix transpose), the involution T(T(A)) = A, the byte multiset,
 * brute force against numpy on every shape up to 8x8, exact Python integer
 * sums, math.fsum within the a-priori error bound of a sequential double sum,
 * and the full 65536-entry decode tables of numpy float16 and torch bfloat16.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

/* Element kinds understood by the oracle (its own numbering). */
enum {
    ORACLE_I32 = 0,
    ORACLE_F32 = 1,
    ORACLE_BF16 = 2,
    ORACLE_F16 = 3
};

/* ------------------------------------------------------------------------ */
/* Transpose, Listing 3.5: out[x][y] = in[y][x].                            */
/* ------------------------------------------------------------------------ */

void oracle_transpose(const void *src, void *dst, int64_t rows, int64_t cols,
                      int64_t esize)
{
    const unsigned char *in = (const unsigned char *)src;
    unsigned char *out = (unsigned char *)dst;
    for (int64_t x = 0; x < cols; x++) {          /* x < W */
        for (int64_t y = 0; y < rows; y++) {      /* y < H */
            /* out[x][y]: row x of the cols x rows output. */
            const unsigned char *from = in + (y * cols + x) * esize;
            unsigned char *to = out + (x * rows + y) * esize;
            for (int64_t b = 0; b < esize; b++)
                to[b] = from[b];
        }
    }
}

/* Listing 3.8: loops by, bx over 32x32 tiles, copy the input tile into a
 * local tile, then write out[bx*32+y][by*32+x] = tile[x][y].  Edge tiles are
 * cut to the matrix. */
void oracle_transpose_tiled(const void *src, void *dst, int64_t rows,
                            int64_t cols, int64_t esize)
{
    const unsigned char *in = (const unsigned char *)src;
    unsigned char *out = (unsigned char *)dst;
    unsigned char tile[32][32][8];
    if (esize > 8)
        return;
    for (int64_t by = 0; by * 32 < rows; by++) {
        for (int64_t bx = 0; bx * 32 < cols; bx++) {
            for (int64_t y = 0; y < 32; y++) {
                for (int64_t x = 0; x < 32; x++) {
                    int64_t r = by * 32 + y, c = bx * 32 + x;
                    if (r < rows && c < cols)
                        memcpy(tile[y][x], in + (r * cols + c) * esize,
                               (size_t)esize);
                }
            }
            for (int64_t y = 0; y < 32; y++) {
                for (int64_t x = 0; x < 32; x++) {
                    int64_t orow = bx * 32 + y, ocol = by * 32 + x;
                    if (orow < cols && ocol < rows)
                        memcpy(out + (orow * rows + ocol) * esize, tile[x][y],
                               (size_t)esize);
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Element decoding, from the format definitions.                          */
/* ------------------------------------------------------------------------ */

/* IEEE-754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction
 * bits.  Exponent 0 encodes zero and subnormals (value = frac * 2^-24),
 * exponent 31 encodes infinities (frac = 0) and NaNs. */
double oracle_decode_f16(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int f = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);
    else if (e == 31)
        v = (f == 0) ? INFINITY : NAN;
    else
        v = ldexp((double)(f + 1024), e - 25);
    return sign ? -v : v;
}

/* bfloat16 is the upper half of an IEEE-754 binary32: placing its 16 bits in
 * the high half of a 32-bit word gives the binary32 with the same value. */
double oracle_decode_bf16(uint16_t b)
{
    uint32_t w = (uint32_t)b << 16;
    float f;
    memcpy(&f, &w, sizeof f);
    return (double)f;
}

static double element_as_double(const void *a, int64_t i, int dtype)
{
    switch (dtype) {
    case ORACLE_I32:
        return (double)((const int32_t *)a)[i];
    case ORACLE_F32:
        return (double)((const float *)a)[i];
    case ORACLE_BF16:
        return oracle_decode_bf16(((const uint16_t *)a)[i]);
    case ORACLE_F16:
        return oracle_decode_f16(((const uint16_t *)a)[i]);
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------------ */
/* Sum, Listing 2.1: sum = 0; for i < N: sum += arr[i].                     */
/* ------------------------------------------------------------------------ */

int64_t oracle_sum_i32(const int32_t *arr, int64_t n)
{
    int64_t sum = 0;
    for (int64_t i = 0; i < n; i++)
        sum += (int64_t)arr[i];
    return sum;
}

double oracle_sum_f64(const void *arr, int64_t n, int dtype)
{
    double sum = 0.0;
    for (int64_t i = 0; i < n; i++)
        sum += element_as_double(arr, i, dtype);
    return sum;
}

/* Neumaier's improvement of Kahan summation (A. Neumaier, "Rundungsfehler-
 * analyse einiger Verfahren zur Summation endlicher Summen", ZAMM 54, 1974):
 * the running sum s is kept with a correction c that collects the low-order
 * bits lost by each addition, whichever operand is larger. */
double oracle_sum_f64_neumaier(const void *arr, int64_t n, int dtype)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double x = element_as_double(arr, i, dtype);
        double t = s + x;
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    return s + c;
}

double oracle_sum_abs_f64(const void *arr, int64_t n, int dtype)
{
    double sum = 0.0;
    for (int64_t i = 0; i < n; i++)
        sum += fabs(element_as_double(arr, i, dtype));
    return sum;
}

/* Listing 2.2: psums[bi] = sum of arr[chunk*bi .. chunk*bi + chunk), then
 * sum = psums[0] + psums[1] + ... in order.  Integer form, exact. */
int64_t oracle_sum_i32_chunked(const int32_t *arr, int64_t n, int64_t chunk)
{
    int64_t sum = 0;
    if (chunk <= 0)
        return 0;
    for (int64_t bi = 0; bi * chunk < n; bi++) {
        int64_t psum = 0;
        for (int64_t i = 0; i < chunk && bi * chunk + i < n; i++)
            psum += (int64_t)arr[bi * chunk + i];
        sum += psum;
    }
    return sum;
}

/* ------------------------------------------------------------------------ */
/* Neighbouring problems (the thesis's Sec. 9 future work and the pitched /  */
/* batched / in-place variants of Listing 3.5).                              */
/* ------------------------------------------------------------------------ */

/* Listing 3.5 on sub-blocks of larger row-major arrays: out[x][y] = in[y][x]
 * with the input row pitch lds and the output row pitch ldd (elements). */
void oracle_transpose_strided(const void *src, int64_t lds, void *dst, int64_t ldd,
                              int64_t rows, int64_t cols, int64_t esize)
{
    const unsigned char *in = (const unsigned char *)src;
    unsigned char *out = (unsigned char *)dst;
    for (int64_t x = 0; x < cols; x++)
        for (int64_t y = 0; y < rows; y++)
            memcpy(out + (x * ldd + y) * esize, in + (y * lds + x) * esize, (size_t)esize);
}

/* Listing 3.5 applied to `batch` dense matrices laid out stride_src (input)
 * and stride_dst (output) elements apart. */
void oracle_transpose_batched(const void *src, int64_t stride_src, void *dst, int64_t stride_dst,
                              int64_t batch, int64_t rows, int64_t cols, int64_t esize)
{
    for (int64_t b = 0; b < batch; b++)
        oracle_transpose((const unsigned char *)src + b * stride_src * esize,
                         (unsigned char *)dst + b * stride_dst * esize, rows, cols, esize);
}

/* In-place transpose of an n x n matrix: swap a[i][j] and a[j][i] for every
 * i < j (the diagonal stays). */
void oracle_transpose_inplace(void *a, int64_t n, int64_t esize)
{
    unsigned char *m = (unsigned char *)a;
    unsigned char t[8];
    if (esize > 8)
        return;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            unsigned char *p = m + (i * n + j) * esize, *q = m + (j * n + i) * esize;
            memcpy(t, p, (size_t)esize);
            memcpy(p, q, (size_t)esize);
            memcpy(q, t, (size_t)esize);
        }
}

/* Inclusive prefix sums, Listing 2.1's loop keeping every intermediate sum:
 * out[i] = A(0) + ... + A(i).  int32 input: exact int64. */
void oracle_scan_i32(const int32_t *arr, int64_t n, int64_t *out)
{
    int64_t sum = 0;
    for (int64_t i = 0; i < n; i++) {
        sum += (int64_t)arr[i];
        out[i] = sum;
    }
}

/* Float input: sequential double prefix sums of the exactly widened values. */
void oracle_scan_f64(const void *arr, int64_t n, int dtype, double *out)
{
    double sum = 0.0;
    for (int64_t i = 0; i < n; i++) {
        sum += element_as_double(arr, i, dtype);
        out[i] = sum;
    }
}

/* Histogram of int32 values: bins of `width` >= 1 integers starting at lo;
 * counts[b] = #{ i : lo + b*width <= x_i < lo + (b+1)*width }, b < nbins.
 * Values outside [lo, lo + nbins*width) are not counted. */
void oracle_histogram_i32(const int32_t *arr, int64_t n, int64_t lo, int64_t width,
                          int64_t nbins, int64_t *counts)
{
    for (int64_t b = 0; b < nbins; b++)
        counts[b] = 0;
    if (width <= 0)
        return;
    for (int64_t i = 0; i < n; i++) {
        int64_t d = (int64_t)arr[i] - lo;
        if (d < 0)
            continue;
        int64_t b = d / width;
        if (b < nbins)
            counts[b] += 1;
    }
}
