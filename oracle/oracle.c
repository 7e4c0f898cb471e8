/*
 * oracle.c -- plain, slow, single-threaded FP64 CPU implementation of the
 * dense stereo-matching path of Zhou & Jagadeesan, "Real-time Dense
 * Reconstruction of Tissue Surface from Stereo Optical Video" (arXiv
 * 2007.12623), Section II.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library: every rule below is written out again from the paper.
 *
 * Everything is computed in double precision, pixel by pixel, straight from
 * the definitions, with no box-sum tricks, blocking or fusion:
 *   - ZNCC is the textbook zero-mean normalised cross-correlation over the
 *     matching window (Sec. II-A), evaluated window by window.
 *   - Winner-take-all picks the best ZNCC among all candidate disparities
 *     (Sec. II-A, "brute force ... test the candidate disparity values").
 *   - Outlier removal, hole filling and their alternation follow Sec. II-B.
 *   - The improved Laplacian refinement follows Sec. II-C, Eqs. (1)-(4).
 * Readings where the paper is silent (tie-breaks, what "sufficient number"
 * and "interpolation" mean, the sub-pixel parabola, the left-right check, the
 * soft-argmin variant) are stated beside each function.
 *
 * Parity pins: every function here is checked by tests/test_oracle_*.py
 * against closed forms, library routines, invariants, hand-derived fixtures
 * under tests/golden/ and finite differences.  Nothing in this file is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ---------------------------------------------------------------- helpers */

static int inside(int W, int H, int x, int y) {
    return x >= 0 && x < W && y >= 0 && y < H;
}

/* Floor division for a possibly negative numerator and a positive
 * denominator. */
static long long floordiv(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* round(num / den) with halves rounded toward +infinity, den > 0:
 * floor((2 num + den) / (2 den)).  Integer-exact. */
static long long round_half_up(long long num, long long den) {
    return floordiv(2 * num + den, 2 * den);
}

/* Window membership.  FULL uses every pixel of the (2r+1)^2 window; the
 * chessboard variant of Sec. II-A uses every other pixel, here the offsets
 * whose dx+dy is even, so the centre pixel is always included. */
static int in_window(int dx, int dy, int sampling) {
    if (sampling == OR_SAMPLE_FULL) return 1;
    return ((dx + dy) % 2) == 0;
}

/* ------------------------------------------------------------------ S0 */

/* RGB (interleaved, 3 bytes per pixel) to 8-bit gray with BT.601 weights in
 * 8-bit fixed point: (77 R + 150 G + 29 B + 128) >> 8.  The paper works on
 * gray ZNCC but does not say how colour video is reduced; this fixed-point
 * rule is the reading taken. */
void or_gray(const uint8_t* rgb, int W, int H, uint8_t* gray) {
    for (int i = 0; i < W * H; ++i) {
        int r = rgb[3 * i + 0], g = rgb[3 * i + 1], b = rgb[3 * i + 2];
        gray[i] = (uint8_t)((77 * r + 150 * g + 29 * b + 128) >> 8);
    }
}

/* ------------------------------------------------------------------ ZNCC */

int or_candidate_valid(int W, int H, int r, int x, int y, int d) {
    /* The whole window must lie inside both images. */
    return y >= r && y < H - r && x >= r && x < W - r && x - d >= r &&
           x - d < W - r;
}

/* ZNCC of the left window centred at (x, y) and the right window centred at
 * (x - d, y) (Sec. II-A).  Returns NaN for an invalid candidate.  A window
 * with zero variance makes the correlation undefined; it is read as 0. */
double or_zncc(const uint8_t* L, const uint8_t* R, int W, int H, int r,
               int sampling, int x, int y, int d) {
    if (!or_candidate_valid(W, H, r, x, y, d)) return NAN;
    double n = 0.0, sl = 0.0, sr = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if (!in_window(dx, dy, sampling)) continue;
            n += 1.0;
            sl += L[(y + dy) * W + (x + dx)];
            sr += R[(y + dy) * W + (x + dx - d)];
        }
    double ml = sl / n, mr = sr / n;
    double cov = 0.0, vl = 0.0, vr = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if (!in_window(dx, dy, sampling)) continue;
            double a = L[(y + dy) * W + (x + dx)] - ml;
            double b = R[(y + dy) * W + (x + dx - d)] - mr;
            cov += a * b;
            vl += a * a;
            vr += b * b;
        }
    if (vl == 0.0 || vr == 0.0) return 0.0;
    return cov / sqrt(vl * vr);
}

/* Full cost volume c = 1 - rho, layout [H][W][D], NaN for invalid
 * candidates. */
void or_cost_volume(const uint8_t* L, const uint8_t* R, int W, int H,
                    int d_min, int D, int r, int sampling, double* cost) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int k = 0; k < D; ++k) {
                double rho = or_zncc(L, R, W, H, r, sampling, x, y, d_min + k);
                cost[((size_t)y * W + x) * D + k] = isnan(rho) ? NAN : 1.0 - rho;
            }
}

/* ------------------------------------------------------- sub-pixel (S3) */

/* Three-point parabola through c(d-1), c(d), c(d+1); returns the offset of
 * its vertex from d, clamped to [-1/2, 1/2], or 0 when the curvature is not
 * positive.  The paper has no sub-pixel step of its own; this is the
 * standard parabola vertex. */
double or_parabola(double cm, double c0, double cp) {
    double den = cm - 2.0 * c0 + cp;
    if (!(den > 0.0)) return 0.0;
    double delta = (cm - cp) / (2.0 * den);
    if (delta > 0.5) delta = 0.5;
    if (delta < -0.5) delta = -0.5;
    return delta;
}

/* ---------------------------------------------------------- WTA (S2-S3) */

/* Winner-take-all for the left pixel (x, y): the candidate with the largest
 * ZNCC; exact ties go to the smallest disparity.  *gap receives the
 * difference between the best and the second-best ZNCC (+inf when there is
 * only one valid candidate); *sub the parabola-refined disparity.  Returns
 * the winning disparity, or OR_INVALID when no candidate is valid. */
int or_wta_left_pixel(const uint8_t* L, const uint8_t* R, int W, int H,
                      int d_min, int D, int r, int sampling, int x, int y,
                      double* gap, double* sub) {
    int best = OR_INVALID;
    double best_rho = -INFINITY, second = -INFINITY;
    for (int k = 0; k < D; ++k) {
        int d = d_min + k;
        double rho = or_zncc(L, R, W, H, r, sampling, x, y, d);
        if (isnan(rho)) continue;
        if (best == OR_INVALID || rho > best_rho) {
            if (best != OR_INVALID) second = best_rho;
            best_rho = rho;
            best = d;
        } else if (rho > second) {
            second = rho;
        }
    }
    if (gap) *gap = (best == OR_INVALID) ? NAN : best_rho - second;
    if (sub) {
        if (best == OR_INVALID) {
            *sub = NAN;
        } else {
            double delta = 0.0;
            if (best > d_min && best < d_min + D - 1) {
                double rm = or_zncc(L, R, W, H, r, sampling, x, y, best - 1);
                double rp = or_zncc(L, R, W, H, r, sampling, x, y, best + 1);
                if (!isnan(rm) && !isnan(rp))
                    delta = or_parabola(1.0 - rm, 1.0 - best_rho, 1.0 - rp);
            }
            *sub = best + delta;
        }
    }
    return best;
}

/* Winner-take-all for the right pixel (u, y): the same ZNCC values, grouped
 * by the right pixel, i.e. the best over d of rho(left = u + d, d).  Ties go
 * to the smallest disparity.  Used by the left-right consistency check. */
int or_wta_right_pixel(const uint8_t* L, const uint8_t* R, int W, int H,
                       int d_min, int D, int r, int sampling, int u, int y,
                       double* gap) {
    int best = OR_INVALID;
    double best_rho = -INFINITY, second = -INFINITY;
    for (int k = 0; k < D; ++k) {
        int d = d_min + k;
        double rho = or_zncc(L, R, W, H, r, sampling, u + d, y, d);
        if (isnan(rho)) continue;
        if (best == OR_INVALID || rho > best_rho) {
            if (best != OR_INVALID) second = best_rho;
            best_rho = rho;
            best = d;
        } else if (rho > second) {
            second = rho;
        }
    }
    if (gap) *gap = (best == OR_INVALID) ? NAN : best_rho - second;
    return best;
}

void or_match(const uint8_t* L, const uint8_t* R, int W, int H, int d_min,
              int D, int r, int sampling, int16_t* dL, int16_t* dR,
              double* sub, double* gapL, double* gapR) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            double g = 0, s = 0, gr = 0;
            int bl = or_wta_left_pixel(L, R, W, H, d_min, D, r, sampling, x, y,
                                       &g, &s);
            int br = or_wta_right_pixel(L, R, W, H, d_min, D, r, sampling, x,
                                        y, &gr);
            if (dL) dL[i] = (int16_t)bl;
            if (dR) dR[i] = (int16_t)br;
            if (sub) sub[i] = s;
            if (gapL) gapL[i] = g;
            if (gapR) gapR[i] = gr;
        }
}

/* ------------------------------------------------------------ LR (S4) */

/* Left-right consistency: a left pixel keeps its disparity d when its right
 * correspondence u = x - d chose a disparity within `thresh` of d.  A left
 * pixel that fails has no corresponding right pixel, i.e. becomes a hole in
 * the sense of Sec. II-B. */
void or_lr_check(const int16_t* dL, const int16_t* dR, int W, int H,
                 int thresh, int16_t* out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            int d = dL[i];
            int keep = 0;
            if (d != OR_INVALID) {
                int u = x - d;
                if (u >= 0 && u < W) {
                    int e = dR[(size_t)y * W + u];
                    if (e != OR_INVALID && abs(d - e) <= thresh) keep = 1;
                }
            }
            out[i] = keep ? (int16_t)d : (int16_t)OR_INVALID;
        }
}

/* ----------------------------------------------- outlier removal (S5) */

static const int DIR8[8][2] = {{1, 0},  {-1, 0}, {0, 1},  {0, -1},
                               {1, 1},  {1, -1}, {-1, 1}, {-1, -1}};

/* Sec. II-B: a valid pixel is kept when at least one of its 8 radial
 * directions, followed for `radius` steps, stays inside the image, meets
 * only valid pixels, and changes disparity by less than `thresh` between
 * every two neighbouring points (starting at the pixel itself).  Otherwise it
 * is an outlier and is removed.  A diagonal step moves one pixel along each
 * axis.  Reads `in`, writes `out` (a Jacobi pass). */
void or_outlier_removal(const int16_t* in, int W, int H, int radius,
                        double thresh, int16_t* out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            if (in[i] == OR_INVALID) {
                out[i] = OR_INVALID;
                continue;
            }
            int keep = 0;
            for (int k = 0; k < 8 && !keep; ++k) {
                int ok = 1;
                int prev = in[i];
                for (int s = 1; s <= radius; ++s) {
                    int qx = x + s * DIR8[k][0], qy = y + s * DIR8[k][1];
                    if (!inside(W, H, qx, qy)) { ok = 0; break; }
                    int v = in[(size_t)qy * W + qx];
                    if (v == OR_INVALID) { ok = 0; break; }
                    if (!(fabs((double)v - (double)prev) < thresh)) { ok = 0; break; }
                    prev = v;
                }
                if (ok) keep = 1;
            }
            out[i] = keep ? in[i] : (int16_t)OR_INVALID;
        }
}

/* ------------------------------------------------- hole filling (S6) */

/* Sec. II-B, first method: a hole searches each of its 8 radial directions
 * up to `radius` steps and takes the first valid pixel met in each.  When
 * at least `min_dirs` directions found one ("sufficient number of
 * neighbouring points"), the hole receives their interpolation, read as the
 * weighted mean with integer weights (radius + 1 - distance), rounded to the
 * nearest integer with halves up, so the filled value stays a discrete
 * disparity (Sec. II-C, first paragraph).  Jacobi: reads `in`, writes
 * `out`. */
void or_fill_radial(const int16_t* in, int W, int H, int radius, int min_dirs,
                    int16_t* out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            out[i] = in[i];
            if (in[i] != OR_INVALID) continue;
            long long num = 0, den = 0;
            int found = 0;
            for (int k = 0; k < 8; ++k) {
                for (int s = 1; s <= radius; ++s) {
                    int qx = x + s * DIR8[k][0], qy = y + s * DIR8[k][1];
                    if (!inside(W, H, qx, qy)) break;
                    int v = in[(size_t)qy * W + qx];
                    if (v != OR_INVALID) {
                        long long w = radius + 1 - s;
                        num += w * v;
                        den += w;
                        found += 1;
                        break;
                    }
                }
            }
            if (found >= min_dirs)
                out[i] = (int16_t)round_half_up(num, den);
        }
}

/* Number of integer offsets (dx, dy) with dx^2 + dy^2 <= radius^2. */
int or_disc_area(int radius) {
    int n = 0;
    for (int dy = -radius; dy <= radius; ++dy)
        for (int dx = -radius; dx <= radius; ++dx)
            if (dx * dx + dy * dy <= radius * radius) ++n;
    return n;
}

/* Sec. II-B, second method: a hole looks at every pixel within `radius`
 * (Euclidean) of itself.  When at least `min_count` of them are valid, it
 * receives their mean, rounded to the nearest integer with halves up.
 * Jacobi: reads `in`, writes `out`. */
void or_fill_disc(const int16_t* in, int W, int H, int radius, int min_count,
                  int16_t* out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            out[i] = in[i];
            if (in[i] != OR_INVALID) continue;
            long long sum = 0, cnt = 0;
            for (int dy = -radius; dy <= radius; ++dy)
                for (int dx = -radius; dx <= radius; ++dx) {
                    if (dx * dx + dy * dy > radius * radius) continue;
                    int qx = x + dx, qy = y + dy;
                    if (!inside(W, H, qx, qy)) continue;
                    int v = in[(size_t)qy * W + qx];
                    if (v == OR_INVALID) continue;
                    sum += v;
                    cnt += 1;
                }
            if (cnt >= min_count && cnt > 0)
                out[i] = (int16_t)round_half_up(sum, cnt);
        }
}

/* Sec. II-B, last paragraph: `rounds` alternations of outlier removal (with
 * radius r0 + t*dr in round t) and hole filling (radial, then disc). */
void or_postprocess(const int16_t* in, int W, int H, int rounds, int r0,
                    int dr, double thresh, int fill_radial_r,
                    int fill_radial_min_dirs, int fill_disc_r,
                    int fill_disc_min_count, int16_t* out) {
    size_t n = (size_t)W * H;
    int16_t* a = (int16_t*)malloc(n * sizeof(int16_t));
    int16_t* b = (int16_t*)malloc(n * sizeof(int16_t));
    memcpy(a, in, n * sizeof(int16_t));
    for (int t = 0; t < rounds; ++t) {
        or_outlier_removal(a, W, H, r0 + t * dr, thresh, b);
        or_fill_radial(b, W, H, fill_radial_r, fill_radial_min_dirs, a);
        or_fill_disc(a, W, H, fill_disc_r, fill_disc_min_count, b);
        memcpy(a, b, n * sizeof(int16_t));
    }
    memcpy(out, a, n * sizeof(int16_t));
    free(a);
    free(b);
}

/* ------------------------------------------- Laplacian refinement (S7) */

/* ZNCC used by the o-update: from the supplied cost volume (c = 1 - rho,
 * [H][W][D], NaN = invalid) when there is one, else computed from the
 * images by the definition above. */
static double refine_rho(const double* cost, const uint8_t* L,
                         const uint8_t* R, int W, int H, int d_min, int D,
                         int r, int sampling, int x, int y, int d) {
    if (d < d_min || d >= d_min + D) return NAN;
    if (cost) {
        double c = cost[((size_t)y * W + x) * D + (d - d_min)];
        return isnan(c) ? NAN : 1.0 - c;
    }
    return or_zncc(L, R, W, H, r, sampling, x, y, d);
}

/* Mean of v over the valid pixels of the (2 rs + 1)^2 box around (x, y)
 * (the box is cut at the image border).  The neighbourhood "within a
 * pre-defined radius" of Eq. (1) is read as this square box, centre
 * included. */
static double box_mean_valid(const double* v, const int16_t* o, int W, int H,
                             int rs, int x, int y) {
    double s = 0.0;
    long n = 0;
    for (int dy = -rs; dy <= rs; ++dy)
        for (int dx = -rs; dx <= rs; ++dx) {
            int qx = x + dx, qy = y + dy;
            if (!inside(W, H, qx, qy)) continue;
            size_t j = (size_t)qy * W + qx;
            if (o[j] == OR_INVALID) continue;
            s += v[j];
            n += 1;
        }
    return s / (double)n;
}

/* Sec. II-C.  o: the discrete disparities after outlier removal and hole
 * filling (OR_INVALID = none).  For k = 1..K on every valid pixel i:
 *   Eq. (1)  dt_i  = mean_j o_j
 *   Eq. (2)  b_i   = dt_i - alpha o_i - (1 - alpha) d_i^(k-1)
 *   Eq. (3)  d_i^k = dt_i - mean_j b_j
 *   Eq. (4)  o_i   = argmin over integer o* in [d_i^k - S, d_i^k + S] of
 *                   1/ZNCC(o*) + eta (o* - d_i^k)^2
 * with d^(0) = o.  Readings: candidates outside the disparity range or with
 * an invalid window are skipped; a non-positive ZNCC makes 1/ZNCC meaningless
 * and is read as an infinite cost; ties go to the smaller |o* - d|, then to
 * the smaller o*; when no candidate is usable o_i is left unchanged.  Invalid
 * pixels stay invalid and get NaN.  Writes d^(K) to d_out and the final o to
 * o_out (either may be NULL). */
void or_refine(const int16_t* o_in, const double* cost, const uint8_t* L,
               const uint8_t* R, int W, int H, int d_min, int D, int r,
               int sampling, int rs, int K, double alpha, double eta,
               int search, double* d_out, int16_t* o_out) {
    size_t n = (size_t)W * H;
    int16_t* o = (int16_t*)malloc(n * sizeof(int16_t));
    double* ov = (double*)malloc(n * sizeof(double));
    double* dprev = (double*)malloc(n * sizeof(double));
    double* dt = (double*)malloc(n * sizeof(double));
    double* b = (double*)malloc(n * sizeof(double));
    double* dk = (double*)malloc(n * sizeof(double));
    memcpy(o, o_in, n * sizeof(int16_t));
    for (size_t i = 0; i < n; ++i) dprev[i] = (o[i] == OR_INVALID) ? NAN : o[i];

    for (int k = 1; k <= K; ++k) {
        for (size_t i = 0; i < n; ++i) ov[i] = (o[i] == OR_INVALID) ? 0.0 : o[i];
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = (size_t)y * W + x;
                if (o[i] == OR_INVALID) continue;
                dt[i] = box_mean_valid(ov, o, W, H, rs, x, y);            /* (1) */
                b[i] = dt[i] - alpha * o[i] - (1.0 - alpha) * dprev[i];  /* (2) */
            }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = (size_t)y * W + x;
                if (o[i] == OR_INVALID) { dk[i] = NAN; continue; }
                dk[i] = dt[i] - box_mean_valid(b, o, W, H, rs, x, y);    /* (3) */
            }
        for (int y = 0; y < H; ++y)                                      /* (4) */
            for (int x = 0; x < W; ++x) {
                size_t i = (size_t)y * W + x;
                if (o[i] == OR_INVALID) continue;
                double d = dk[i];
                int lo = (int)ceil(d - search), hi = (int)floor(d + search);
                int best = OR_INVALID;
                double best_f = INFINITY, best_dist = INFINITY;
                for (int c = lo; c <= hi; ++c) {
                    double rho = refine_rho(cost, L, R, W, H, d_min, D, r,
                                            sampling, x, y, c);
                    if (isnan(rho) || !(rho > 0.0)) continue;
                    double f = 1.0 / rho + eta * (c - d) * (c - d);
                    double dist = fabs(c - d);
                    if (best == OR_INVALID || f < best_f ||
                        (f == best_f && dist < best_dist)) {
                        best = c;
                        best_f = f;
                        best_dist = dist;
                    }
                }
                if (best != OR_INVALID) o[i] = (int16_t)best;
            }
        memcpy(dprev, dk, n * sizeof(double));
    }
    if (d_out) memcpy(d_out, dprev, n * sizeof(double));
    if (o_out) memcpy(o_out, o, n * sizeof(int16_t));
    free(o); free(ov); free(dprev); free(dt); free(b); free(dk);
}

/* ---------------------------------------------------- whole path */

void or_pipeline(const uint8_t* L, const uint8_t* R, int W, int H,
                 const or_params* p, int16_t* dL, int16_t* dR, double* sub,
                 int16_t* o_lr, int16_t* o_post, double* d_final,
                 double* cost_out) {
    size_t n = (size_t)W * H;
    int16_t* l = dL ? dL : (int16_t*)malloc(n * sizeof(int16_t));
    int16_t* rr = dR ? dR : (int16_t*)malloc(n * sizeof(int16_t));
    int16_t* lr = o_lr ? o_lr : (int16_t*)malloc(n * sizeof(int16_t));
    int16_t* pp = o_post ? o_post : (int16_t*)malloc(n * sizeof(int16_t));
    double* cost = cost_out ? cost_out
                            : (double*)malloc(n * (size_t)p->num_disp * sizeof(double));
    or_cost_volume(L, R, W, H, p->d_min, p->num_disp, p->win_radius,
                   p->sampling, cost);
    or_match(L, R, W, H, p->d_min, p->num_disp, p->win_radius, p->sampling, l,
             rr, sub, NULL, NULL);
    or_lr_check(l, rr, W, H, p->lr_thresh, lr);
    or_postprocess(lr, W, H, p->outlier_rounds, p->r0, p->dr,
                   p->outlier_thresh, p->fill_radial_r, p->fill_radial_min_dirs,
                   p->fill_disc_r, p->fill_disc_min_count, pp);
    or_refine(pp, cost, L, R, W, H, p->d_min, p->num_disp, p->win_radius,
              p->sampling, p->smooth_radius, p->smooth_iters, p->alpha,
              p->eta, p->refine_search, d_final, NULL);
    if (!dL) free(l);
    if (!dR) free(rr);
    if (!o_lr) free(lr);
    if (!o_post) free(pp);
    if (!cost_out) free(cost);
}

/* ------------------------------------------- soft-argmin (S8, S9) */

/* ZNCC on real-valued images together with what its gradient needs. */
typedef struct {
    double rho, ml, mr, vl, vr, n;
    int degenerate;
} zstat;

static int zncc_f(const double* L, const double* R, int W, int H, int r,
                  int sampling, int x, int y, int d, zstat* z) {
    if (!or_candidate_valid(W, H, r, x, y, d)) return 0;
    double n = 0.0, sl = 0.0, sr = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if (!in_window(dx, dy, sampling)) continue;
            n += 1.0;
            sl += L[(y + dy) * W + (x + dx)];
            sr += R[(y + dy) * W + (x + dx - d)];
        }
    double ml = sl / n, mr = sr / n;
    double cov = 0.0, vl = 0.0, vr = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            if (!in_window(dx, dy, sampling)) continue;
            double a = L[(y + dy) * W + (x + dx)] - ml;
            double b = R[(y + dy) * W + (x + dx - d)] - mr;
            cov += a * b;
            vl += a * a;
            vr += b * b;
        }
    z->n = n; z->ml = ml; z->mr = mr; z->vl = vl; z->vr = vr;
    z->degenerate = (vl == 0.0 || vr == 0.0);
    z->rho = z->degenerate ? 0.0 : cov / sqrt(vl * vr);
    return 1;
}

/* Soft-argmin disparity (not in the paper; the differentiable variant):
 * p_d = softmax over the valid candidates of rho_d / tau, d_soft = sum d p_d.
 * Also returns the log-sum-exp of the logits.  Pixels without a valid
 * candidate get NaN and has_valid = 0. */
void or_softargmin_fwd(const double* L, const double* R, int W, int H,
                       int d_min, int D, int r, int sampling, double tau,
                       double* dsoft, double* lse, uint8_t* has_valid) {
    double* z = (double*)malloc((size_t)D * sizeof(double));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            double m = -INFINITY;
            int any = 0;
            for (int k = 0; k < D; ++k) {
                zstat s;
                if (zncc_f(L, R, W, H, r, sampling, x, y, d_min + k, &s)) {
                    z[k] = s.rho / tau;
                    if (z[k] > m) m = z[k];
                    any = 1;
                } else {
                    z[k] = NAN;
                }
            }
            if (!any) {
                dsoft[i] = NAN;
                if (lse) lse[i] = NAN;
                if (has_valid) has_valid[i] = 0;
                continue;
            }
            double se = 0.0;
            for (int k = 0; k < D; ++k)
                if (!isnan(z[k])) se += exp(z[k] - m);
            double l = m + log(se);
            double ds = 0.0;
            for (int k = 0; k < D; ++k)
                if (!isnan(z[k])) ds += (d_min + k) * exp(z[k] - l);
            dsoft[i] = ds;
            if (lse) lse[i] = l;
            if (has_valid) has_valid[i] = 1;
        }
    free(z);
}

/* Gradient of sum_i grad_dsoft[i] * d_soft[i] with respect to both images.
 * Chain rule: d d_soft / d rho_d = p_d (d - d_soft) / tau; and for the left
 * window pixel q (right pixel q - d) of a non-degenerate window,
 *   d rho / d L(q)   = (R(q-d) - mr) / sqrt(vl vr) - rho (L(q) - ml) / vl
 *   d rho / d R(q-d) = (L(q) - ml) / sqrt(vl vr) - rho (R(q-d) - mr) / vr
 * (the derivatives through the window means vanish because centred values
 * sum to zero).  A degenerate window (zero variance) has rho fixed at 0 and
 * contributes nothing. */
void or_softargmin_bwd(const double* L, const double* R, int W, int H,
                       int d_min, int D, int r, int sampling, double tau,
                       const double* grad_dsoft, double* gL, double* gR) {
    size_t n = (size_t)W * H;
    memset(gL, 0, n * sizeof(double));
    memset(gR, 0, n * sizeof(double));
    double* dsoft = (double*)malloc(n * sizeof(double));
    double* lse = (double*)malloc(n * sizeof(double));
    uint8_t* hv = (uint8_t*)malloc(n);
    or_softargmin_fwd(L, R, W, H, d_min, D, r, sampling, tau, dsoft, lse, hv);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            if (!hv[i] || grad_dsoft[i] == 0.0) continue;
            for (int k = 0; k < D; ++k) {
                int d = d_min + k;
                zstat s;
                if (!zncc_f(L, R, W, H, r, sampling, x, y, d, &s)) continue;
                if (s.degenerate) continue;
                double p = exp(s.rho / tau - lse[i]);
                double G = grad_dsoft[i] * p * (d - dsoft[i]) / tau;
                double a = 1.0 / sqrt(s.vl * s.vr);
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        if (!in_window(dx, dy, sampling)) continue;
                        size_t ql = (size_t)(y + dy) * W + (x + dx);
                        size_t qr = (size_t)(y + dy) * W + (x + dx - d);
                        double lc = L[ql] - s.ml, rc = R[qr] - s.mr;
                        gL[ql] += G * (a * rc - s.rho * lc / s.vl);
                        gR[qr] += G * (a * lc - s.rho * rc / s.vr);
                    }
            }
        }
    free(dsoft);
    free(lse);
    free(hv);
}

/* L1 loss of the soft-argmin disparity against a reference field:
 * mean over pixels with a valid candidate of |d_soft - gt|, and its
 * gradient sign(d_soft - gt) / |V| (sign(0) = 0; 0 off V). */
double or_l1_loss(const double* dsoft, const uint8_t* has_valid,
                  const double* gt, size_t n, double* grad) {
    size_t nv = 0;
    for (size_t i = 0; i < n; ++i) nv += has_valid[i] ? 1 : 0;
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!has_valid[i] || nv == 0) {
            if (grad) grad[i] = 0.0;
            continue;
        }
        double e = dsoft[i] - gt[i];
        s += fabs(e);
        if (grad) grad[i] = (e > 0 ? 1.0 : (e < 0 ? -1.0 : 0.0)) / (double)nv;
    }
    return nv ? s / (double)nv : 0.0;
}

/* Disparity -> 3-D points in the left rectified camera frame, the
 * reprojection of a calibrated rectified pair (Sec. II: physical depths are
 * computed directly from the disparities after calibration, equivalently to
 * Matlab's reconstructScene):
 *     Z = f B / (d + doffs),  X = (u - cx) Z / f,  Y = (v - cy) Z / f,
 * with doffs = right principal point minus left principal point.  NaN (all
 * three coordinates) where d is NaN or d + doffs <= 0.
 * Normals: the cross product of the central differences
 *     (P(u+1,v) - P(u-1,v)) x (P(u,v+1) - P(u,v-1)),
 * turned to face the camera (n . P <= 0) and normalised; NaN where one of
 * the four neighbours is missing (image border or NaN point) or the cross
 * product vanishes.  xyz and nrm are [H][W][3]; either may be NULL. */
void or_depth_points(const double* d, int W, int H, double f, double cx, double cy,
                     double B, double doffs, double* xyz, double* nrm) {
    const double nan = NAN;
    double* P = (double*)malloc(sizeof(double) * 3 * (size_t)W * H);
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            double* p = P + 3 * ((size_t)v * W + u);
            const double dv = d[(size_t)v * W + u];
            if (isnan(dv) || !(dv + doffs > 0.0)) {
                p[0] = p[1] = p[2] = nan;
                continue;
            }
            const double Z = f * B / (dv + doffs);
            p[0] = (u - cx) * Z / f;
            p[1] = (v - cy) * Z / f;
            p[2] = Z;
        }
    if (xyz) memcpy(xyz, P, sizeof(double) * 3 * (size_t)W * H);
    if (nrm) {
        for (int v = 0; v < H; ++v)
            for (int u = 0; u < W; ++u) {
                double* n = nrm + 3 * ((size_t)v * W + u);
                n[0] = n[1] = n[2] = nan;
                if (u < 1 || u > W - 2 || v < 1 || v > H - 2) continue;
                const double* pc = P + 3 * ((size_t)v * W + u);
                const double* pl = P + 3 * ((size_t)v * W + u - 1);
                const double* pr = P + 3 * ((size_t)v * W + u + 1);
                const double* pu = P + 3 * ((size_t)(v - 1) * W + u);
                const double* pd = P + 3 * ((size_t)(v + 1) * W + u);
                if (isnan(pc[2]) || isnan(pl[2]) || isnan(pr[2]) || isnan(pu[2]) || isnan(pd[2])) continue;
                const double a[3] = {pr[0] - pl[0], pr[1] - pl[1], pr[2] - pl[2]};
                const double b[3] = {pd[0] - pu[0], pd[1] - pu[1], pd[2] - pu[2]};
                double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
                const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                if (!(len > 0.0)) continue;
                double s = 1.0 / len;
                if (c[0] * pc[0] + c[1] * pc[1] + c[2] * pc[2] > 0.0) s = -s;
                n[0] = c[0] * s;
                n[1] = c[1] * s;
                n[2] = c[2] * s;
            }
    }
    free(P);
}

/* ------------------------------------------------------------------------
 * Point-based TSDF mosaicking of one key frame into the surface model
 * (Sec. II, GPU-based TSDF mosaicking).  The model is a list of points with
 * a world position, an RGB colour, a position weight and a colour weight.
 * Every quantity below is evaluated in double precision.
 *
 *  1. Rasterise the model into the current image: X = R P + t (world ->
 *     camera); a point with X.z > 0 lands on pixel u = floor(f X.x / X.z + cx
 *     + 1/2), v = floor(f X.y / X.z + cy + 1/2); per pixel the nearest point
 *     (smallest X.z, ties -> smallest index) is kept.
 *  2. Every pixel with a valid stereo point Q (camera frame) whose kept
 *     model point lies within the truncation distance (|Q.z - X.z| <= tau)
 *     merges into it: P <- (w P + Pw) / (w + 1), w <- w + 1 with Pw = R^T
 *     (Q - t), and C <- (c C + g I) / (c + g), c <- c + g, where I is the
 *     pixel's colour and g its colour weight: 1 inside the central disc
 *     (normalised radius rr <= r0, rr = 1 at the corners), falling linearly
 *     to gmin at the corners.
 *  3. Every other pixel with a valid point is appended as a new point
 *     (Pw, I, w = 1, c = g), in row-major pixel order, while capacity lasts.
 * Returns the number of appends that did not fit (0 normally).
 * pos/rgb: [capacity][3]; wpos/wrgb: [capacity]; *count in/out.
 *
 * Decision margins (optional outputs, NULL to skip).  A computation in a
 * narrower precision may decide differently where a decision lies within
 * its rounding of an edge; the oracle marks those places:
 *   fragile_pix[W*H]: pixel k is marked when a point's projection lies
 *     within eps_pix pixels of a rounding edge (u + 1/2 or v + 1/2 within
 *     eps_pix of an integer; the pixels on both sides are marked), when the
 *     two nearest points of k differ in depth by at most eps_rel times the
 *     nearer depth, or when k's merge test is within eps_rel * (|Q.z| + tau)
 *     of its threshold;
 *   fragile_pt[n]: model point i is marked when its projection is near an
 *     edge or it lands on a marked pixel;
 *   src_pixel[capacity]: for every appended point, the pixel it came from. */
static void or_mark(uint8_t* fp, int W, int H, double fu, double fv) {
    if (fu >= 0.0 && fu < (double)W && fv >= 0.0 && fv < (double)H) fp[(size_t)fv * W + (size_t)fu] = 1;
}

int or_mosaic_frame(double* pos, double* rgb, double* wpos, double* wrgb, int* count, int capacity,
                    const float* xyz, const uint8_t* img, int W, int H, float f, float cx, float cy,
                    const float* R, const float* t, float tau, float r0, float gmin,
                    double eps_pix, double eps_rel, uint8_t* fragile_pix, uint8_t* fragile_pt, int* src_pixel) {
    const int n = *count;
    const size_t np = (size_t)W * H;
    int* win = (int*)malloc(sizeof(int) * np);
    double* winz = (double*)malloc(sizeof(double) * np);
    double* z2nd = (double*)malloc(sizeof(double) * np);   /* second-nearest depth per pixel */
    long long* land = (long long*)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    double Rd[9], td[3];
    for (int a = 0; a < 9; ++a) Rd[a] = R[a];
    for (int a = 0; a < 3; ++a) td[a] = t[a];
    for (size_t k = 0; k < np; ++k) {
        win[k] = -1;
        z2nd[k] = INFINITY;
    }
    if (fragile_pix) memset(fragile_pix, 0, np);
    if (fragile_pt) memset(fragile_pt, 0, (size_t)n);
    for (int i = 0; i < n; ++i) {
        land[i] = -1;
        const double* P = pos + 3 * (size_t)i;
        double X[3];
        for (int a = 0; a < 3; ++a) X[a] = Rd[3 * a] * P[0] + Rd[3 * a + 1] * P[1] + Rd[3 * a + 2] * P[2] + td[a];
        if (!(X[2] > 0.0)) continue;
        const double pu = (double)f * X[0] / X[2] + (double)cx + 0.5;
        const double pv = (double)f * X[1] / X[2] + (double)cy + 0.5;
        const double fu = floor(pu), fv = floor(pv);
        if (fragile_pix) {
            /* near a rounding edge: mark the pixel and its neighbour across the edge */
            const double eu = pu - fu, ev = pv - fv;
            int near_edge = 0;
            if (eu < eps_pix) { or_mark(fragile_pix, W, H, fu - 1, fv); near_edge = 1; }
            if (eu > 1.0 - eps_pix) { or_mark(fragile_pix, W, H, fu + 1, fv); near_edge = 1; }
            if (ev < eps_pix) { or_mark(fragile_pix, W, H, fu, fv - 1); near_edge = 1; }
            if (ev > 1.0 - eps_pix) { or_mark(fragile_pix, W, H, fu, fv + 1); near_edge = 1; }
            if (near_edge) {
                or_mark(fragile_pix, W, H, fu, fv);
                if (fragile_pt) fragile_pt[i] = 1;
            }
        }
        if (!(fu >= 0.0 && fu < (double)W && fv >= 0.0 && fv < (double)H)) continue;
        const size_t k = (size_t)fv * W + (size_t)fu;
        land[i] = (long long)k;
        if (win[k] < 0 || X[2] < winz[k]) {     /* equal depth: the smaller index stays */
            if (win[k] >= 0) z2nd[k] = winz[k];
            win[k] = i;
            winz[k] = X[2];
        } else if (X[2] < z2nd[k]) {
            z2nd[k] = X[2];
        }
    }
    if (fragile_pix)
        for (size_t k = 0; k < np; ++k)
            if (win[k] >= 0 && z2nd[k] - winz[k] <= eps_rel * winz[k]) fragile_pix[k] = 1;
    const double cxc = (W - 1) / 2.0, cyc = (H - 1) / 2.0;
    int appended = 0, dropped = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            const size_t k = (size_t)v * W + u;
            const double Qx = xyz[3 * k], Qy = xyz[3 * k + 1], Qz = xyz[3 * k + 2];
            if (isnan(Qz) || !(Qz > 0.0)) continue;
            /* world point R^T (Q - t) */
            const double q0 = Qx - td[0], q1 = Qy - td[1], q2 = Qz - td[2];
            double Pw[3];
            for (int a = 0; a < 3; ++a) Pw[a] = Rd[a] * q0 + Rd[3 + a] * q1 + Rd[6 + a] * q2;
            const double du = (u - cxc) / (W / 2.0), dv = (v - cyc) / (H / 2.0);
            const double rr = sqrt(du * du + dv * dv) / sqrt(2.0);
            double g = 1.0;
            if (rr > r0) g = 1.0 - (1.0 - gmin) * (rr - r0) / (1.0 - r0);
            if (g < gmin) g = gmin;
            const int i = win[k];
            if (i >= 0 && fragile_pix && fabs(fabs(Qz - winz[k]) - (double)tau) <= eps_rel * (fabs(Qz) + tau))
                fragile_pix[k] = 1;
            if (i >= 0 && fabs(Qz - winz[k]) <= (double)tau) {
                const double w = wpos[i], c = wrgb[i];
                for (int a = 0; a < 3; ++a) {
                    pos[3 * (size_t)i + a] = (w * pos[3 * (size_t)i + a] + Pw[a]) / (w + 1.0);
                    rgb[3 * (size_t)i + a] = (c * rgb[3 * (size_t)i + a] + g * img[3 * k + a]) / (c + g);
                }
                wpos[i] = w + 1.0;
                wrgb[i] = c + g;
                continue;
            }
            if (n + appended >= capacity) { ++dropped; continue; }
            const size_t j = (size_t)(n + appended);
            for (int a = 0; a < 3; ++a) {
                pos[3 * j + a] = Pw[a];
                rgb[3 * j + a] = img[3 * k + a];
            }
            wpos[j] = 1.0;
            wrgb[j] = g;
            if (src_pixel) src_pixel[j] = (int)k;
            ++appended;
        }
    if (fragile_pt && fragile_pix)
        for (int i = 0; i < n; ++i)
            if (land[i] >= 0 && fragile_pix[land[i]]) fragile_pt[i] = 1;
    *count = n + appended;
    free(win);
    free(winz);
    free(z2nd);
    free(land);
    return dropped;
}

/* ------------------------------------------------------------------------
 * Histogram-voting preselection of feature-match inliers (Sec. II,
 * histogram voting-based matching inliers preselection): correct matches
 * between adjacent frames share nearly the same displacement (du, dv) =
 * (u2 - u1, v2 - v1).  Displacements are binned into a 2-D histogram of
 * bins of side `bin` over [-range, range)^2 (bin index floor((du + range) /
 * bin), single precision; a displacement outside the range votes for no
 * bin); the score of a match is the histogram count summed over the 3x3
 * bins around its own (0 outside the range), and the matches are ranked by
 * score, higher first, ties by index.  hist: nb x nb counts (nb =
 * ceil(2 range / bin)); score, order: n entries. */
static const int* or_vote_score_ptr;
static int or_vote_cmp(const void* a, const void* b) {
    const int i = *(const int*)a, j = *(const int*)b;
    if (or_vote_score_ptr[i] != or_vote_score_ptr[j]) return or_vote_score_ptr[i] > or_vote_score_ptr[j] ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

int or_vote_nbins(float bin, float range) {
    return (int)ceilf((2.0f * range) / bin);
}

void or_vote_matches(const float* uv1, const float* uv2, int n, float bin, float range, int* hist,
                     int* score, int* order) {
    const int nb = or_vote_nbins(bin, range);
    int* bx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* by = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < nb * nb; ++k) hist[k] = 0;
    for (int i = 0; i < n; ++i) {
        const float du = uv2[2 * i] - uv1[2 * i], dv = uv2[2 * i + 1] - uv1[2 * i + 1];
        const float fx = floorf((du + range) / bin), fy = floorf((dv + range) / bin);
        bx[i] = by[i] = -1;
        if (fx >= 0.0f && fx < (float)nb && fy >= 0.0f && fy < (float)nb) {
            bx[i] = (int)fx;
            by[i] = (int)fy;
            hist[by[i] * nb + bx[i]] += 1;
        }
    }
    for (int i = 0; i < n; ++i) {
        int s = 0;
        if (bx[i] >= 0)
            for (int y = by[i] - 1; y <= by[i] + 1; ++y)
                for (int x = bx[i] - 1; x <= bx[i] + 1; ++x)
                    if (x >= 0 && x < nb && y >= 0 && y < nb) s += hist[y * nb + x];
        score[i] = s;
        order[i] = i;
    }
    or_vote_score_ptr = score;
    qsort(order, (size_t)n, sizeof(int), or_vote_cmp);
    free(bx);
    free(by);
}
