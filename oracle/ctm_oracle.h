/*
 * ctm_oracle.h -- plain CPU oracle for object-centric Census Template Matching
 * (arXiv 2604.07980, Sec. 4.3 and Algorithm 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg (and its
 * `--impl reference` arm) may load it.  It shares no code, header, table or
 * helper with the CUDA path and never calls it.
 *
 * Every routine is the literal definition written as loops: per-pixel census
 * (Sec. 4.3.1, Algorithm 1), the Hamming cost sum (Eq. census_cost) for every
 * candidate, first argmin, parabola (Eq. subpixel), the backward search
 * (Sec. 4.3.3), occlusion-aware sampling (Sec. 4.3.5), sorted-segment
 * aggregation (Sec. 4.3.4) and Eq. 1.  No blocking, fusion or reordering.
 */
#ifndef CTM_ORACLE_H
#define CTM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Matching parameters.  Field meaning is identical to the CUDA library's
 * parameter block (the two are declared independently). */
typedef struct {
    int32_t win_w, win_h;      /* census window (odd sizes); win_w*win_h + sentinel <= 64 */
    int32_t sentinel;          /* 1: leading 1 bit above the comparison bits (Algorithm 1) */
    int32_t far_side_px;       /* tau_s: FAR iff max(w, h) < tau_s (clipped, full-res px)  */
    int32_t close_factor;      /* k: CLOSE boxes match on the census of I(k x, k y)         */
    int32_t far_dmin, far_dmax;       /* FAR disparity range, full-res px                  */
    int32_t close_dmin, close_dmax;   /* CLOSE disparity range, px of the scaled grid      */
    int32_t dy_min, dy_max;    /* vertical search range (both passes)                     */
    int32_t grid_g;            /* CLOSE box -> g x g blocks                               */
    int32_t pts_side;          /* at most pts_side x pts_side sampled points per block    */
    int32_t min_pts;           /* a block needs >= min_pts usable points                  */
    int32_t fb_tol;            /* forward-backward accept iff |d_b - d_f| <= fb_tol       */
    float   agg_tau_d;         /* run: consecutive sorted differences < tau_d (full-res)  */
    int32_t agg_nmin;          /* run must hold >= N_min blocks                           */
    int32_t agg_mode;          /* 0 = median of the run, 1 = trimmed mean of the run      */
    float   trim_frac;         /* trimmed mean drops floor(trim_frac*m) from each end     */
    int32_t max_occluders;     /* keep at most this many occluders per box                */
    float   frontal_crop;      /* 0: occluders ranked nearest first; c in (0, 1]: those
                                  whose clipped box centre lies in the centred crop of
                                  c W x c H rank first (each group nearest first)      */
} orc_params;

/* Per-block result (one per box x block slot; FAR boxes use slot 0). */
typedef struct {
    int32_t n_pts;     /* sampled grid points (nx*ny)                                 */
    int32_t n_valid;   /* points used: census defined in L and not inside an occluder */
    int32_t d_f, dy_f; /* forward first argmin                                        */
    int32_t d_b, dy_b; /* backward first argmin                                       */
    int32_t s_m, s_0, s_p; /* forward costs at (dy_f, d_f-1), (dy_f, d_f), (dy_f, d_f+1)
                              (s_m/s_p are 0 when outside the range)                   */
    float   d_sub;     /* parabola-refined disparity on the matching grid             */
    float   d_full;    /* d_sub * k, full-resolution px                               */
    int32_t flags;     /* ORC_BLK_* bits                                              */
} orc_block;

enum {
    ORC_BLK_VALID = 1,          /* enough points and forward-backward consistent */
    ORC_BLK_FB_REJECT = 2,      /* |d_b - d_f| > fb_tol                          */
    ORC_BLK_FEW_POINTS = 4,     /* n_valid < min_pts (no search run)             */
    ORC_BLK_SUBPIX_CLAMPED = 8, /* d_f at a range end: no parabola offset        */
    ORC_BLK_PRESENT = 16        /* the slot is a real block of this box          */
};

enum {
    ORC_BOX_VALID = 1,
    ORC_BOX_FB_REJECT = 2,
    ORC_BOX_FEW_POINTS = 4,
    ORC_BOX_NO_SEGMENT = 8,
    ORC_BOX_NONPOS_DISP = 16,
    ORC_BOX_EMPTY = 32,
    ORC_BOX_SUBPIX_CLAMPED = 64,
    ORC_BOX_FAR = 128
};

/* Census (Sec. 4.3.1, Algorithm 1) of the decimated image I_k(x, y) = I(k x, k y),
 * which is I itself for k = 1.  out is Ws*Hs codes, Ws = ceil(W/k), Hs = ceil(H/k),
 * row-major without padding.  Pixels whose window leaves the decimated image get 0. */
void orc_census(const uint8_t *img, int W, int H, int pitch, int k,
                int win_w, int win_h, int sentinel, uint64_t *out);

/* Eq. subpixel on three integer costs around an interior argmin. */
float orc_subpixel(int d_star, int32_t s_m, int32_t s_0, int32_t s_p);

/* Sec. 4.3.4 robust aggregation of n block disparities (any order).
 * Returns 1 and writes *out when a run of >= nmin blocks exists, else 0. */
int orc_aggregate(const float *vals, int n, float tau_d, int nmin, int mode,
                  float trim_frac, float *out);

/* Eq. 1: Z = f b / d (fp32; f*b formed once).  NaN for d <= 0. */
float orc_depth(float f_px, float baseline_m, float d);

/* Algorithm 2 for one frame.  boxes: n x {x0, y0, x1, y1, frame} half-open
 * full-res rectangles (frame is ignored).  disp/depth/flags: n entries.
 * blk (optional): n * slots entries, slots = max(1, grid_g^2).
 * cost_f / cost_b (optional): n * slots * NC int32, NC = max over FAR/CLOSE of
 * (dmax-dmin+1)*(dy_max-dy_min+1); candidate c = (dy-dy_min)*N_d + (d-dmin).
 * Returns 0 on success, negative on invalid arguments. */
int orc_match_frame(const uint8_t *L, const uint8_t *R, int W, int H, int pitch,
                    const int32_t *boxes, int n, float f_px, float baseline_m,
                    const orc_params *p, float *disp, float *depth, uint8_t *flags,
                    orc_block *blk, int32_t *cost_f, int32_t *cost_b);

/* Camera geometry of one frame for orc_box_points. */
typedef struct {
    double Q[16];        /* 4x4 row-major reprojection matrix: [X Y Z W]^T = Q [u v d 1]^T */
    double T[12];        /* 3x4 row-major camera-to-vehicle transform [R | t]               */
    double disp_var;     /* sigma_d^2 (px^2), the configured disparity variance            */
    double f_px, baseline_m;
    int32_t width, height;   /* image size: boxes are clipped to it                        */
} orc_geometry;

/* Sec. 4.3.6 disparity-to-depth conversion and covariance estimation, in
 * double, for n boxes after matching.  Box i uses geo[boxes[i].frame].  For a
 * VALID box: (u, v) = centre of the clipped box in pixel coordinates (pixel c
 * spans [c, c+1), its centre is c; so u = (x0 + x1 - 1) / 2), d = disp[i];
 * [X Y Z W] = Q [u v d 1]; p = (X, Y, Z) / W; p_v = R p + t;
 * sigma_Z^2 = Z^4 sigma_d^2 / (f^2 b^2) with Z = p.z.  out[8 i ..]: p.x, p.y,
 * p.z, p_v.x, p_v.y, p_v.z, sigma_Z^2, W; all NaN when the box is not VALID,
 * its frame index is outside [0, n_geo) or W == 0.  The paper prints no
 * worked example; the tests pin this against closed forms. */
void orc_box_points(const int32_t *boxes, const float *disp, const uint8_t *flags, int n,
                    const orc_geometry *geo, int n_geo, double *out);

/* Sec. 5.1 auto-rectification offset, with census matching in place of BM.
 * For every delta in [delta_min, delta_max] and every pixel (x, y) of the ROI
 * [rx0, rx1) x [ry0, ry1): the left image is read shifted down by delta rows
 * (left pixel (x, y + delta)); d_f = first argmin over d in [dmin, dmax] of
 * popcount(C_L(x, y + delta) ^ C_R(x - d, y)); the backward search from the
 * right pixel q = (x - d_f, y) gives d_b = first argmin over d' of
 * popcount(C_R(q) ^ C_L(q.x + d', y + delta)); the pixel counts when its left
 * census is defined (window inside the image), |d_b - d_f| <= fb_tol and
 * d_f > d_thresh.  Codes outside
 * the image read as 0 (as in the box search).  counts[i] = the count for
 * delta_min + i; returns delta* = the first delta with the largest count. */
int orc_auto_rect(const uint8_t *L, const uint8_t *R, int W, int H, int pitch, int win_w, int win_h,
                  int sentinel, int rx0, int ry0, int rx1, int ry1, int dmin, int dmax, int delta_min,
                  int delta_max, int d_thresh, int fb_tol, int64_t *counts);

/* Temporal filter of the per-frame estimates (Sec. 5.1): delta_t = median of the
 * last n estimates (n >= 1; even n: the lower of the middle two), and the step
 * from prev is clamped to [-max_step, max_step].  Returns prev + clamped step. */
int orc_rect_filter(const int *estimates, int n, int prev, int max_step);

#ifdef __cplusplus
}
#endif
#endif
