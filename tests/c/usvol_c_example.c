/* The nearest-neighbour path driven from plain C through include/usvol.h:
 * device memory from cudaMalloc, no Python and no PyTorch.
 *
 *   usvol_c_example <input> <output>
 *
 * input  (little-endian, written by tests/test_gpu_c_abi.py):
 *   int32 n, H, W, nx, ny, nz, z_lo, z_hi
 *   float64 spacing[3], origin[3], sx, sy, calibration[16]
 *   float64 poses[n][16], uint8 images[n][H][W]
 * output: float32 projection[ny][nx], uint16 counts[ny][nx]
 * Exit status 0 on success; a failing call prints its name and message. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "usvol.h"

#define CHECK_USV(call)                                                            \
    do {                                                                           \
        int rc_ = (call);                                                          \
        if (rc_ != USV_OK) {                                                       \
            fprintf(stderr, "%s: %s (%s)\n", #call, usv_strerror(rc_),             \
                    usv_last_cuda_error());                                        \
            return 1;                                                              \
        }                                                                          \
    } while (0)

#define CHECK_CUDA(call)                                                           \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));           \
            return 1;                                                              \
        }                                                                          \
    } while (0)

static int read_all(FILE *f, void *p, size_t n)
{
    return fread(p, 1, n, f) == n ? 0 : -1;
}

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s <input> <output>\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in)
        return 2;
    int32_t hdr[8];
    double spacing[3], origin[3], sx, sy;
    usv_calibration cal;
    memset(&cal, 0, sizeof(cal));
    if (read_all(in, hdr, sizeof(hdr)) || read_all(in, spacing, sizeof(spacing)) ||
        read_all(in, origin, sizeof(origin)) || read_all(in, &sx, 8) || read_all(in, &sy, 8) ||
        read_all(in, cal.image_to_probe, sizeof(cal.image_to_probe)))
        return 2;
    const int32_t n = hdr[0], H = hdr[1], W = hdr[2];
    const usv_grid grid = {hdr[3], hdr[4], hdr[5]};
    const int32_t z_lo = hdr[6], z_hi = hdr[7];
    const size_t frame_bytes = (size_t)n * H * W, pose_bytes = (size_t)n * 16 * sizeof(double);
    const size_t plane = (size_t)grid.nx * grid.ny;
    double *poses = (double *)malloc(pose_bytes);
    uint8_t *images = (uint8_t *)malloc(frame_bytes);
    if (!poses || !images || read_all(in, poses, pose_bytes) || read_all(in, images, frame_bytes))
        return 2;
    fclose(in);
    cal.geom = USV_LINEAR;
    cal.sx_mm = sx;
    cal.sy_mm = sy;

    const size_t bytes = usv_volume_bytes(grid, USV_PNN);
    if (bytes == 0)
        return 2;
    void *storage = NULL, *d_images = NULL, *d_out = NULL, *d_cnt = NULL;
    CHECK_CUDA(cudaMalloc(&storage, bytes));
    CHECK_CUDA(cudaMalloc(&d_images, frame_bytes));
    CHECK_CUDA(cudaMalloc(&d_out, plane * sizeof(float)));
    CHECK_CUDA(cudaMalloc(&d_cnt, plane * sizeof(uint16_t)));
    CHECK_CUDA(cudaMemcpy(d_images, images, frame_bytes, cudaMemcpyHostToDevice));

    cudaStream_t st;
    CHECK_CUDA(cudaStreamCreate(&st));
    usv_volume *vol = NULL;
    CHECK_USV(usv_volume_create(grid, spacing, origin, USV_PNN, storage, bytes, &vol));
    CHECK_USV(usv_volume_reset(vol, st));
    /* poses straight from host memory: the library stages them */
    CHECK_USV(usv_insert_frames(vol, d_images, n, H, W, USV_U8, poses, &cal, st));
    CHECK_USV(usv_fill_holes(vol, 1, st));
    CHECK_USV(usv_project_depth_band(vol, z_lo, z_hi, (float *)d_out, (uint16_t *)d_cnt, st));
    const int status = usv_status(vol, st);  /* waits for the stream */
    if (status != 0) {
        fprintf(stderr, "device status %d\n", status);
        return 1;
    }

    float *out = (float *)malloc(plane * sizeof(float));
    uint16_t *cnt = (uint16_t *)malloc(plane * sizeof(uint16_t));
    if (!out || !cnt)
        return 2;
    CHECK_CUDA(cudaMemcpy(out, d_out, plane * sizeof(float), cudaMemcpyDeviceToHost));
    CHECK_CUDA(cudaMemcpy(cnt, d_cnt, plane * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    FILE *o = fopen(argv[2], "wb");
    if (!o || fwrite(out, sizeof(float), plane, o) != plane ||
        fwrite(cnt, sizeof(uint16_t), plane, o) != plane)
        return 2;
    fclose(o);

    CHECK_USV(usv_volume_destroy(vol));
    cudaStreamDestroy(st);
    cudaFree(storage);
    cudaFree(d_images);
    cudaFree(d_out);
    cudaFree(d_cnt);
    free(poses);
    free(images);
    free(out);
    free(cnt);
    return 0;
}
