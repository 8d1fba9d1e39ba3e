/* A plain C client of the librearr C ABI that moves data on the GPU: device
 * buffers from the CUDA runtime (cudaMalloc), one rearr_permute of a 2 x 3
 * fp32 matrix into its 3 x 2 transpose (Sec. III.B, a 2-D transpose), and
 * the result checked here against the transpose written out by hand.
 * Prints "device_permute OK" or what went wrong, for tests/test_c_abi.py. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "librearr.h"

int main(void)
{
    const float a[6] = {1.0f, 2.0f, 3.0f,   /* row 0 */
                        4.0f, 5.0f, 6.0f};  /* row 1 */
    const float want[6] = {1.0f, 4.0f,      /* column 0 of a */
                           2.0f, 5.0f,      /* column 1 */
                           3.0f, 6.0f};     /* column 2 */
    float got[6];
    void *src = NULL, *dst = NULL;
    if (cudaMalloc(&src, sizeof a) != cudaSuccess || cudaMalloc(&dst, sizeof a) != cudaSuccess) {
        printf("device_permute cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(src, a, sizeof a, cudaMemcpyHostToDevice);
    cudaMemset(dst, 0xFF, sizeof a);
    const int64_t dims[2] = {2, 3};
    const int perm[2] = {1, 0};
    rearr_status st = rearr_permute(dst, src, sizeof(float), 2, dims, perm, (rearr_stream_t)0);
    if (st != REARR_OK) {
        printf("device_permute %s %s\n", rearr_status_str(st), rearr_last_error());
        return 1;
    }
    if (cudaMemcpy(got, dst, sizeof got, cudaMemcpyDeviceToHost) != cudaSuccess) {
        printf("device_permute copy-back failed\n");
        return 1;
    }
    cudaFree(src);
    cudaFree(dst);
    if (memcmp(got, want, sizeof got) != 0) {
        printf("device_permute MISMATCH %g %g %g %g %g %g\n", got[0], got[1], got[2], got[3], got[4], got[5]);
        return 1;
    }
    printf("device_permute OK\n");
    return 0;
}
