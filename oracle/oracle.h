/*
 * oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see oracle.c).  This header belongs to the oracle alone and is not
 * included by the CUDA library.
 */
#ifndef STEREO_ORACLE_H
#define STEREO_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#define OR_INVALID (-32768)
#define OR_SAMPLE_FULL 0
#define OR_SAMPLE_CHESSBOARD 1

typedef struct {
    int d_min, num_disp, win_radius, sampling;
    int lr_thresh;
    int outlier_rounds, r0, dr;
    double outlier_thresh;
    int fill_radial_r, fill_radial_min_dirs;
    int fill_disc_r, fill_disc_min_count;
    int smooth_radius, smooth_iters;
    double alpha, eta;
    int refine_search;
} or_params;

void or_gray(const uint8_t* rgb, int W, int H, uint8_t* gray);
int or_candidate_valid(int W, int H, int r, int x, int y, int d);
double or_zncc(const uint8_t* L, const uint8_t* R, int W, int H, int r,
               int sampling, int x, int y, int d);
void or_cost_volume(const uint8_t* L, const uint8_t* R, int W, int H,
                    int d_min, int D, int r, int sampling, double* cost);
double or_parabola(double cm, double c0, double cp);
int or_wta_left_pixel(const uint8_t* L, const uint8_t* R, int W, int H,
                      int d_min, int D, int r, int sampling, int x, int y,
                      double* gap, double* sub);
int or_wta_right_pixel(const uint8_t* L, const uint8_t* R, int W, int H,
                       int d_min, int D, int r, int sampling, int u, int y,
                       double* gap);
void or_match(const uint8_t* L, const uint8_t* R, int W, int H, int d_min,
              int D, int r, int sampling, int16_t* dL, int16_t* dR,
              double* sub, double* gapL, double* gapR);
void or_lr_check(const int16_t* dL, const int16_t* dR, int W, int H,
                 int thresh, int16_t* out);
void or_outlier_removal(const int16_t* in, int W, int H, int radius,
                        double thresh, int16_t* out);
void or_fill_radial(const int16_t* in, int W, int H, int radius, int min_dirs,
                    int16_t* out);
int or_disc_area(int radius);
void or_fill_disc(const int16_t* in, int W, int H, int radius, int min_count,
                  int16_t* out);
void or_postprocess(const int16_t* in, int W, int H, int rounds, int r0,
                    int dr, double thresh, int fill_radial_r,
                    int fill_radial_min_dirs, int fill_disc_r,
                    int fill_disc_min_count, int16_t* out);
void or_refine(const int16_t* o_in, const double* cost, const uint8_t* L,
               const uint8_t* R, int W, int H, int d_min, int D, int r,
               int sampling, int rs, int K, double alpha, double eta,
               int search, double* d_out, int16_t* o_out);
void or_pipeline(const uint8_t* L, const uint8_t* R, int W, int H,
                 const or_params* p, int16_t* dL, int16_t* dR, double* sub,
                 int16_t* o_lr, int16_t* o_post, double* d_final,
                 double* cost_out);
void or_softargmin_fwd(const double* L, const double* R, int W, int H,
                       int d_min, int D, int r, int sampling, double tau,
                       double* dsoft, double* lse, uint8_t* has_valid);
void or_softargmin_bwd(const double* L, const double* R, int W, int H,
                       int d_min, int D, int r, int sampling, double tau,
                       const double* grad_dsoft, double* gL, double* gR);
double or_l1_loss(const double* dsoft, const uint8_t* has_valid,
                  const double* gt, size_t n, double* grad);
void or_depth_points(const double* d, int W, int H, double f, double cx, double cy,
                     double B, double doffs, double* xyz, double* nrm);
int or_vote_nbins(float bin, float range);
void or_vote_matches(const float* uv1, const float* uv2, int n, float bin, float range, int* hist,
                     int* score, int* order);
int or_mosaic_frame(double* pos, double* rgb, double* wpos, double* wrgb, int* count, int capacity,
                    const float* xyz, const uint8_t* img, int W, int H, float f, float cx, float cy,
                    const float* R, const float* t, float tau, float r0, float gmin,
                    double eps_pix, double eps_rel, uint8_t* fragile_pix, uint8_t* fragile_pt, int* src_pixel);

#endif
