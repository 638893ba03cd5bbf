/*
 * CPU oracle for single-precision GEMM -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code; the library's compute path never does.
 *
 * It computes the plain definition of the operation the paper tunes
 * (Section V-B: "GEMM operations" over the (M, N, K) input grid; the BLAS
 * statement of GEMM):
 *
 *     C_ref[i][j] = alpha * sum_{k<K} op(A)[i][k] * op(B)[k][j] + beta * C_in[i][j]
 *
 * from the same FP32 inputs the GPU sees, with every product and every sum
 * carried in FP64.  The product of two FP32 numbers is exact in FP64
 * (24 + 24 significand bits <= 53), so the only roundings are those of the
 * FP64 additions.  Loop order is i-k-j (row i of the result is accumulated
 * over k into an FP64 row buffer); OpenMP splits the rows.  beta == 0 means
 * C_in is not read (BLAS convention), so NaNs in C_in do not propagate.
 *
 * Row-major storage: op(A) is M x K and op(B) is K x N.
 *   transA == 'N': A is M x K, element (i,k) at A[i*lda + k]
 *   transA == 'T': A is K x M, element (i,k) at A[k*lda + i]
 *   transB == 'N': B is K x N, element (k,j) at B[k*ldb + j]
 *   transB == 'T': B is N x K, element (k,j) at B[j*ldb + k]
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double op_a(char t, const float *A, long lda, long i, long k)
{
    return (double)((t == 'N') ? A[i * lda + k] : A[k * lda + i]);
}

static double op_b(char t, const float *B, long ldb, long k, long j)
{
    return (double)((t == 'N') ? B[k * ldb + j] : B[j * ldb + k]);
}

/*
 * Computes the rows listed in rows[0..nrows) (all M rows when rows == NULL)
 * into out (FP64, row r of out at out[r*ldo], r indexing the list).
 * C_in (row-major, leading dimension ldc) is read only when beta != 0.
 * Returns 0, or -1 on an invalid argument / allocation failure.
 */
int oracle_gemm_f64(char transA, char transB, long M, long N, long K,
                    double alpha, const float *A, long lda,
                    const float *B, long ldb, double beta,
                    const float *C_in, long ldc,
                    double *out, long ldo, const long *rows, long nrows)
{
    long count = rows ? nrows : M;
    int bad = 0;
    if ((transA != 'N' && transA != 'T') || (transB != 'N' && transB != 'T'))
        return -1;
    if (M < 0 || N < 0 || K < 0 || ldo < N)
        return -1;
    if (count == 0 || N == 0)
        return 0;

#pragma omp parallel
    {
        double *acc = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
        if (!acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long r = 0; r < count; ++r) {
            if (!acc)
                continue;
            long i = rows ? rows[r] : r;
            memset(acc, 0, (size_t)N * sizeof(double));
            for (long k = 0; k < K; ++k) {
                double a = op_a(transA, A, lda, i, k);
                for (long j = 0; j < N; ++j)
                    acc[j] += a * op_b(transB, B, ldb, k, j);
            }
            double *o = out + r * ldo;
            for (long j = 0; j < N; ++j) {
                double v = alpha * acc[j];
                if (beta != 0.0)
                    v += beta * (double)C_in[i * ldc + j];
                o[j] = v;
            }
        }
        free(acc);
    }
    return bad ? -1 : 0;
}

/* Number of OpenMP threads a parallel region of the oracle will use. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Caps the oracle's thread count (n >= 1); no effect without OpenMP. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}
