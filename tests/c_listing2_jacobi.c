/* A C host program in the style of the paper's Listing 2 (Sec. 4, Jacobi), written against the
 * library's C ABI with the paper's variadic calls: it partitions a 2-D binary64 array by rows,
 * applies the two Jacobi kernels (the step, then the copy back) for a number of iterations, reads
 * the array back and writes it, row-major, to a binary file.
 *
 *   c_listing2_jacobi <dpath file: the number of logical devices> <n> <iterations> <output file>
 *
 * The input is the n x n field u[i][j] = ((i * 31 + j * 17) % 101) / 101 with a zero boundary ring. */
#include <stdio.h>
#include <stdlib.h>

#define HDARRAY_SHORT_NAMES /* the paper's ROW, SUM, ... */
#include "hdarray.h"

int main(int argc, char *argv[])
{
    if (argc != 5) {
        fprintf(stderr, "usage: %s dpath n iterations out\n", argv[0]);
        return 2;
    }
    const int n = atoi(argv[2]), iters = atoi(argv[3]);
    double *u = (double *)calloc((size_t)n * n, sizeof(double));
    if (!u || n < 3) return 2;
    for (int i = 1; i < n - 1; i++)
        for (int j = 1; j < n - 1; j++) u[(size_t)i * n + j] = (double)((i * 31 + j * 17) % 101) / 101.0;

    if (HDArrayInit(argc, argv, NULL, argv[1]) < 0) return 3;
    HDArray_t *B = HDArrayCreate("B", "double", u, 2, n, n);
    HDArray_t *A = HDArrayCreate("A", "double", u, 2, n, n);
    const int data = HDArrayPartition(ROW, 2, n, n, 0, 0, n, n);          /* whole array */
    const int work = HDArrayPartition(ROW, 2, n, n, 1, 1, n - 1, n - 1);  /* interior */
    if (!B || !A || data < 0 || work < 0) return 4;
    HDArrayWrite(B, u, data);
    HDArrayWrite(A, u, data);
    for (int t = 0; t < iters; t++) {
        HDArrayApplyKernel("jacobi2d", work, B, A);  /* A = 4-neighbour mean of B */
        HDArrayApplyKernel("copy", work, A, B);      /* B = A */
    }
    HDArrayRead(B, u, data);
    double sum = 0.0;
    HDArrayReduce(B, &sum, SUM, work);
    const int err = HDArrayGetLastError();
    HDArrayExit();
    if (err) {
        fprintf(stderr, "library error %d\n", err);
        return 5;
    }
    FILE *f = fopen(argv[4], "wb");
    if (!f || fwrite(u, sizeof(double), (size_t)n * n, f) != (size_t)n * n) return 6;
    fclose(f);
    printf("%.17g\n", sum);
    free(u);
    return 0;
}
