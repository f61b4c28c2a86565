/* CPU oracle for the free-hand ultrasound volume path (test infrastructure
 * only; see usv_oracle.c).  Shares nothing with the CUDA library. */
#ifndef USV_ORACLE_H
#define USV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int convex;        /* 0: linear probe, 1: convex fan */
    double sx, sy;     /* linear: pixel spacing (mm) lateral / axial */
    double r0, dr;     /* convex: first radius, radial step (mm) */
    double sector_deg; /* convex: full sector angle */
} ora_geometry;

int ora_set_threads(int n);
int64_t ora_round_half_away(double x);
int ora_frame_affine_q32(const double P[16], const double K[16], double sx, double sy,
                         const double spacing[3], const double origin[3], int64_t coef[9]);
int64_t ora_insert_pnn(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                       const uint8_t *images, int n, int H, int W, const double *poses,
                       const double K[16], double sx, double sy,
                       const double spacing[3], const double origin[3]);
void ora_fill_pnn(const uint64_t *sum, const uint32_t *cnt, int nx, int ny, int nz,
                  uint8_t *val, uint8_t *has);
void ora_project_u8(const uint8_t *val, const uint8_t *has, int nx, int ny, int nz, int lo,
                    int hi, float *out, uint16_t *cnt);
int64_t ora_insert_trilinear(double *S, double *Wt, int nx, int ny, int nz,
                             const void *images, int is_f32, int n, int H, int W,
                             const double *poses, const double K[16], const ora_geometry *g,
                             const double spacing[3], const double origin[3]);
void ora_fill_trilinear(const double *S, const double *Wt, int nx, int ny, int nz, double *val,
                        uint8_t *has);
int64_t ora_insert_pnn_rows(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                            const uint8_t *images, int n, int H, int W, const double *poses,
                            const double K[16], double sx, double sy,
                            const double spacing[3], const double origin[3],
                            const int32_t *first_rows);
int64_t ora_insert_pnn_rows_mt(uint64_t *sum, uint32_t *cnt, int nx, int ny, int nz,
                               const uint8_t *images, int n, int H, int W, const double *poses,
                               const double K[16], double sx, double sy,
                               const double spacing[3], const double origin[3],
                               const int32_t *first_rows);
int64_t ora_insert_trilinear_rows(double *S, double *Wt, int nx, int ny, int nz,
                                  const void *images, int is_f32, int n, int H, int W,
                                  const double *poses, const double K[16],
                                  const ora_geometry *g, const double spacing[3],
                                  const double origin[3], const int32_t *first_rows);
void ora_cut_rows_alg1(const double *poses, int n, int H, const double K[16], double k,
                       double d_mm, double l_mm, const double e[3], const double p1[3],
                       double row_mm, int32_t *rows, double *cut_mm);
void ora_bone_rows_alg2(const uint8_t *images, int n, int H, int W, int from, int drop,
                        int window, int margin, int32_t *bone, int32_t *rows);
void ora_project_f64(const double *val, const uint8_t *has, int nx, int ny, int nz, int lo,
                     int hi, double *out, uint16_t *cnt);

#ifdef __cplusplus
}
#endif
#endif
