/*
 * ctm_oracle.c -- plain CPU oracle for object-centric Census Template Matching
 * (arXiv 2604.07980, Sec. 4.3, Algorithm 2).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  It shares nothing with the CUDA library.
 *
 * Written as the definitions, one loop per sum, in the order Algorithm 2 gives:
 *   census at both resolutions -> classify each box FAR/CLOSE -> sample points,
 *   excluding occluded ones -> match FAR blocks, then CLOSE blocks (forward
 *   search, backward search, consistency test, parabola) -> FAR disparity from its
 *   block, CLOSE disparity by robust aggregation -> depth by Eq. 1.
 *
 * Readings of points the paper leaves open are stated where they are used.
 * Pins: Fig. 2's printed census code, the
 * invariants the paper states, closed forms and brute force on tiny inputs
 * (tests/test_oracle_*.py).
 */
#include "ctm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Census, Sec. 4.3.1 and Algorithm 1                                          */
/* ------------------------------------------------------------------------ */

/* xi(a, b) = 1 iff a > b (strict), Sec. 4.3.1. */
static int xi(int a, int b) { return a > b ? 1 : 0; }

/* Census of the decimated image I_k(x, y) = I(k x, k y) (Sec. 4.3.1: at a
 * reduced census size the source coordinates are scaled; with an integer
 * factor k that is plain decimation).  Bits are shifted in raster order of the
 * window (row j outer, column i inner), the order Fig. 2 prints them; the first
 * neighbour ends up in the highest comparison bit.  The centre's own bit (always
 * 0) is kept, because the concatenation in the census equation runs over all
 * (i, j) including (0, 0).  With the sentinel, Algorithm 1 starts the code at 1,
 * so a defined pixel always carries the bit just above the comparison bits.
 * A pixel whose window leaves the image is undefined and stored as 0. */
void orc_census(const uint8_t *img, int W, int H, int pitch, int k,
                int win_w, int win_h, int sentinel, uint64_t *out)
{
    int Ws = (W + k - 1) / k, Hs = (H + k - 1) / k;
    int sx = win_w / 2, sy = win_h / 2;
    for (int y = 0; y < Hs; ++y) {
        for (int x = 0; x < Ws; ++x) {
            uint64_t c;
            if (x - sx < 0 || x + sx >= Ws || y - sy < 0 || y + sy >= Hs) {
                out[(size_t)y * Ws + x] = 0;
                continue;
            }
            int centre = img[(size_t)(k * y) * pitch + (size_t)(k * x)];
            c = sentinel ? 1u : 0u;
            for (int j = -sy; j <= sy; ++j) {
                for (int i = -sx; i <= sx; ++i) {
                    int v = img[(size_t)(k * (y + j)) * pitch + (size_t)(k * (x + i))];
                    c = (c << 1) | (uint64_t)xi(v, centre);
                }
            }
            out[(size_t)y * Ws + x] = c;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. subpixel, Eq. 1 and the robust aggregation of Sec. 4.3.4               */
/* ------------------------------------------------------------------------ */

/* Eq. subpixel: d_hat = d* - (S(d*+1) - S(d*-1)) / (2 (S(d*+1) + S(d*-1) - 2 S(d*))).
 * Eq. census_cost writes the search in dx with the right pixel at x + dx; the
 * library searches d = -dx (right pixel at x - d), and the vertex formula has the
 * same form in d because a parabola's vertex offset flips sign with its axis.
 * fp32 with one IEEE division; costs are exact integers in fp32. */
float orc_subpixel(int d_star, int32_t s_m, int32_t s_0, int32_t s_p)
{
    float num = (float)(s_p - s_m);
    float den = 2.0f * (float)(s_p + s_m - 2 * s_0);
    if (den == 0.0f) return (float)d_star;
    float off = num / den;
    return (float)d_star - off;
}

/* Eq. 1, Z = f b / d.  f*b is formed in fp32 first, then one division. */
float orc_depth(float f_px, float baseline_m, float d)
{
    float fb = f_px * baseline_m;
    if (!(d > 0.0f)) return NAN;
    return fb / d;
}

static void sort_floats(float *v, int n)
{
    /* insertion sort, ascending */
    for (int i = 1; i < n; ++i) {
        float t = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
        v[j + 1] = t;
    }
}

/* Sec. 4.3.4: sort the block disparities; find the longest run whose
 * consecutive differences are all below tau_d (strict); require at least N_min
 * members; return the median of the run (mode 0) or its trimmed mean (mode 1).
 * Equal-length runs: the first one met scanning upward.  Even-length median:
 * mean of the two middle values, (a + b) * 0.5.  Trimmed mean: drop
 * floor(trim_frac * m) values from each end, sum the rest in ascending order. */
int orc_aggregate(const float *vals, int n, float tau_d, int nmin, int mode,
                  float trim_frac, float *out)
{
    if (n <= 0) return 0;
    float *v = (float *)malloc(sizeof(float) * (size_t)n);
    memcpy(v, vals, sizeof(float) * (size_t)n);
    sort_floats(v, n);

    int best_start = 0, best_len = 1;
    int cur_start = 0, cur_len = 1;
    for (int i = 1; i < n; ++i) {
        if (v[i] - v[i - 1] < tau_d) {
            cur_len += 1;
        } else {
            cur_start = i;
            cur_len = 1;
        }
        if (cur_len > best_len) { best_len = cur_len; best_start = cur_start; }
    }
    if (best_len < nmin) { free(v); return 0; }

    const float *run = v + best_start;
    int m = best_len;
    float r;
    if (mode == 0) {
        if (m % 2 == 1) r = run[m / 2];
        else r = (run[m / 2 - 1] + run[m / 2]) * 0.5f;
    } else {
        int t = (int)floorf(trim_frac * (float)m);
        int cnt = m - 2 * t;
        float s = 0.0f;
        for (int i = t; i < m - t; ++i) s += run[i];
        r = s / (float)cnt;
    }
    free(v);
    *out = r;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct { int x0, y0, x1, y1; } rect_t;

static int rect_empty(rect_t r) { return r.x1 <= r.x0 || r.y1 <= r.y0; }

static int rects_overlap(rect_t a, rect_t b)
{
    /* positive-area intersection of half-open rectangles */
    int ix0 = a.x0 > b.x0 ? a.x0 : b.x0, ix1 = a.x1 < b.x1 ? a.x1 : b.x1;
    int iy0 = a.y0 > b.y0 ? a.y0 : b.y0, iy1 = a.y1 < b.y1 ? a.y1 : b.y1;
    return ix1 > ix0 && iy1 > iy0;
}

static int inside(rect_t r, int x, int y) { return x >= r.x0 && x < r.x1 && y >= r.y0 && y < r.y1; }

static int ceil_div(int a, int b) { return (a + b - 1) / b; } /* a >= 0, b > 0 */

/* Priority rule of Sec. 4.3.5 when there are more occluders than slots: an
 * occluder is frontal if its clipped box centre lies in the centred crop
 * [W (1 - c) / 2, W (1 + c) / 2) x [H (1 - c) / 2, H (1 + c) / 2); compared on
 * doubled coordinates, x0 + x1 against W (1 - c) and W (1 + c), in fp32. */
static int frontal(rect_t q, int W, int H, float c)
{
    if (!(c > 0.0f)) return 0;
    const float sx = (float)(q.x0 + q.x1), sy = (float)(q.y0 + q.y1);
    return sx >= (float)W * (1.0f - c) && sx < (float)W * (1.0f + c) &&
           sy >= (float)H * (1.0f - c) && sy < (float)H * (1.0f + c);
}

/* 1 if occluder a ranks before occluder b: frontal first, then larger bottom y,
 * then lower index. */
static int occluder_before(int a, int b, const rect_t *cb, int W, int H, float c)
{
    const int fa = frontal(cb[a], W, H, c), fb = frontal(cb[b], W, H, c);
    if (fa != fb) return fa > fb;
    if (cb[a].y1 != cb[b].y1) return cb[a].y1 > cb[b].y1;
    return a < b;
}

/* Code of a census plane at (x, y); positions outside the plane read as 0, the
 * same value an undefined census pixel holds. */
static uint64_t code_at(const uint64_t *c, int Ws, int Hs, int x, int y)
{
    if (x < 0 || x >= Ws || y < 0 || y >= Hs) return 0;
    return c[(size_t)y * Ws + x];
}

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

/* Eq. census_cost with d = -dx:  S(dy, d) = sum_p popc(C_L(p) xor C_R(p.x - d, p.y + dy)). */
static int32_t cost_forward(const uint64_t *CL, const uint64_t *CR, int Ws, int Hs,
                            const int *px, const int *py, int np, int d, int dy)
{
    int32_t s = 0;
    for (int t = 0; t < np; ++t)
        s += popc64(code_at(CL, Ws, Hs, px[t], py[t]) ^
                    code_at(CR, Ws, Hs, px[t] - d, py[t] + dy));
    return s;
}

/* Sec. 4.3.3 backward pass: the query is the right-image census at the matched
 * position q = (p.x - d_f, p.y + dy_f); the left image is searched at
 * (q.x + d', q.y - dy') over the same ranges. */
static int32_t cost_backward(const uint64_t *CL, const uint64_t *CR, int Ws, int Hs,
                             const int *px, const int *py, int np, int d_f, int dy_f,
                             int d, int dy)
{
    int32_t s = 0;
    for (int t = 0; t < np; ++t) {
        int qx = px[t] - d_f, qy = py[t] + dy_f;
        s += popc64(code_at(CR, Ws, Hs, qx, qy) ^ code_at(CL, Ws, Hs, qx + d, qy - dy));
    }
    return s;
}

static int params_ok(const orc_params *p)
{
    if (p->win_w < 1 || p->win_h < 1 || (p->win_w % 2) == 0 || (p->win_h % 2) == 0) return 0;
    if (p->win_w * p->win_h + (p->sentinel ? 1 : 0) > 64) return 0;
    if (p->close_factor < 1) return 0;
    if (p->far_dmin > p->far_dmax || p->close_dmin > p->close_dmax) return 0;
    if (p->dy_min > p->dy_max) return 0;
    if (p->grid_g < 1 || p->pts_side < 1 || p->min_pts < 1) return 0;
    if (p->fb_tol < 0 || p->agg_nmin < 1 || p->max_occluders < 0) return 0;
    if (!(p->frontal_crop >= 0.0f && p->frontal_crop <= 1.0f)) return 0;
    if (p->agg_mode != 0 && p->agg_mode != 1) return 0;
    if (!(p->trim_frac >= 0.0f && p->trim_frac < 0.5f)) return 0;
    return 1;
}

int orc_match_frame(const uint8_t *L, const uint8_t *R, int W, int H, int pitch,
                    const int32_t *boxes, int n, float f_px, float baseline_m,
                    const orc_params *p, float *disp, float *depth, uint8_t *flags,
                    orc_block *blk, int32_t *cost_f, int32_t *cost_b)
{
    if (!L || !R || W < 1 || H < 1 || pitch < W || n < 0 || !p || !params_ok(p)) return -1;
    if (n > 0 && (!boxes || !disp || !depth || !flags)) return -1;

    const int k_close = p->close_factor;
    const int slots = p->grid_g * p->grid_g;
    const int ndy = p->dy_max - p->dy_min + 1;
    const int nd_far = p->far_dmax - p->far_dmin + 1;
    const int nd_close = p->close_dmax - p->close_dmin + 1;
    const int nc_max = (nd_far > nd_close ? nd_far : nd_close) * ndy;

    /* Algorithm 2, first step: census images at the original and the scaled resolution. */
    const int W1 = W, H1 = H;
    const int Wk = ceil_div(W, k_close), Hk = ceil_div(H, k_close);
    uint64_t *CL1 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W1 * H1);
    uint64_t *CR1 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W1 * H1);
    uint64_t *CLk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)Wk * Hk);
    uint64_t *CRk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)Wk * Hk);
    orc_census(L, W, H, pitch, 1, p->win_w, p->win_h, p->sentinel, CL1);
    orc_census(R, W, H, pitch, 1, p->win_w, p->win_h, p->sentinel, CR1);
    orc_census(L, W, H, pitch, k_close, p->win_w, p->win_h, p->sentinel, CLk);
    orc_census(R, W, H, pitch, k_close, p->win_w, p->win_h, p->sentinel, CRk);

    /* Boxes are clipped to the image first; everything below uses clipped boxes. */
    rect_t *cb = (rect_t *)malloc(sizeof(rect_t) * (size_t)(n > 0 ? n : 1));
    int *is_far = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const int32_t *b = boxes + 5 * (size_t)i;
        rect_t r;
        r.x0 = b[0] < 0 ? 0 : b[0];
        r.y0 = b[1] < 0 ? 0 : b[1];
        r.x1 = b[2] > W ? W : b[2];
        r.y1 = b[3] > H ? H : b[3];
        if (rect_empty(r)) { r.x0 = r.y0 = r.x1 = r.y1 = 0; }
        cb[i] = r;
        /* Sec. 4.3.4 classification: FAR iff the larger side in full-res px < tau_s. */
        int w = r.x1 - r.x0, h = r.y1 - r.y0;
        int side = w > h ? w : h;
        is_far[i] = side < p->far_side_px;
    }

    if (blk) memset(blk, 0, sizeof(orc_block) * (size_t)n * slots);
    if (cost_f) memset(cost_f, 0, sizeof(int32_t) * (size_t)n * slots * nc_max);
    if (cost_b) memset(cost_b, 0, sizeof(int32_t) * (size_t)n * slots * nc_max);

    int *px = (int *)malloc(sizeof(int) * (size_t)p->pts_side * p->pts_side);
    int *py = (int *)malloc(sizeof(int) * (size_t)p->pts_side * p->pts_side);
    int32_t *Sf = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc_max);
    int32_t *Sb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nc_max);
    int *occ = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    orc_block *bres = (orc_block *)malloc(sizeof(orc_block) * (size_t)slots);
    float *dvals = (float *)malloc(sizeof(float) * (size_t)slots);

    /* Algorithm 2 batches FAR blocks, then CLOSE blocks; pass 0 = FAR, pass 1 = CLOSE. */
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < n; ++i) {
            if ((pass == 0) != (is_far[i] != 0)) continue;
            rect_t r = cb[i];
            const int far = is_far[i];
            const int k = far ? 1 : k_close;
            const int g = far ? 1 : p->grid_g;
            const int dmin = far ? p->far_dmin : p->close_dmin;
            const int dmax = far ? p->far_dmax : p->close_dmax;
            const int nd = dmax - dmin + 1;
            const int Ws = far ? W1 : Wk, Hs = far ? H1 : Hk;
            const uint64_t *CL = far ? CL1 : CLk;
            const uint64_t *CR = far ? CR1 : CRk;
            int fb_any = 0, few_any = 0, clamp_any = 0;
            uint8_t fl = far ? ORC_BOX_FAR : 0;

            disp[i] = NAN;
            depth[i] = NAN;

            /* The box on the matching grid: decimated pixel x belongs to the box iff
             * its source pixel k x does, i.e. x in [ceil(x0/k), ceil(x1/k)). */
            int sx0 = ceil_div(r.x0, k), sx1 = ceil_div(r.x1, k);
            int sy0 = ceil_div(r.y0, k), sy1 = ceil_div(r.y1, k);
            if (rect_empty(r) || sx1 <= sx0 || sy1 <= sy0) {
                flags[i] = (uint8_t)(fl | ORC_BOX_EMPTY);
                continue;
            }

            /* Sec. 4.3.5: B_j occludes B_i iff they overlap and B_j's bottom y is
             * larger.  At most max_occluders are kept: frontal ones first (box
             * centre inside the centred crop, when frontal_crop > 0), then the
             * others, each group nearest first (largest bottom y), ties by index. */
            int nocc = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (rects_overlap(r, cb[j]) && cb[j].y1 > r.y1) occ[nocc++] = j;
            }
            for (int a = 1; a < nocc; ++a) { /* insertion sort: frontal, bottom desc, index asc */
                int t = occ[a], b = a - 1;
                while (b >= 0 && occluder_before(t, occ[b], cb, W, H, p->frontal_crop)) {
                    occ[b + 1] = occ[b];
                    --b;
                }
                occ[b + 1] = t;
            }
            if (nocc > p->max_occluders) nocc = p->max_occluders;

            const int bw = sx1 - sx0, bh = sy1 - sy0;
            for (int s = 0; s < g * g; ++s) {
                orc_block *o = &bres[s];
                memset(o, 0, sizeof(*o));
                o->flags = ORC_BLK_PRESENT;
                int a = s % g, bb = s / g; /* blocks in row-major order */
                int bx0 = sx0 + (a * bw) / g, bx1 = sx0 + ((a + 1) * bw) / g;
                int by0 = sy0 + (bb * bh) / g, by1 = sy0 + ((bb + 1) * bh) / g;
                int nx = bx1 - bx0 < p->pts_side ? bx1 - bx0 : p->pts_side;
                int ny = by1 - by0 < p->pts_side ? by1 - by0 : p->pts_side;
                o->n_pts = nx * ny;

                /* Sec. 4.3.4 regular point grid: nx x ny points centred in their
                 * cells; a point is used when its left census is defined and its
                 * full-res position lies in no kept occluder (Sec. 4.3.5). */
                int np = 0;
                const int sxw = p->win_w / 2, syw = p->win_h / 2;
                for (int m = 0; m < ny; ++m) {
                    int y = by0 + ((2 * m + 1) * (by1 - by0)) / (2 * ny);
                    for (int q = 0; q < nx; ++q) {
                        int x = bx0 + ((2 * q + 1) * (bx1 - bx0)) / (2 * nx);
                        if (x - sxw < 0 || x + sxw >= Ws || y - syw < 0 || y + syw >= Hs) continue;
                        int hidden = 0;
                        for (int t = 0; t < nocc; ++t)
                            if (inside(cb[occ[t]], k * x, k * y)) { hidden = 1; break; }
                        if (hidden) continue;
                        px[np] = x;
                        py[np] = y;
                        ++np;
                    }
                }
                o->n_valid = np;
                if (np < p->min_pts) {
                    o->flags |= ORC_BLK_FEW_POINTS;
                    few_any = 1;
                    continue;
                }

                /* Forward search (Eq. census_cost, exhaustive) and first argmin in
                 * the order (dy ascending, d ascending). */
                int best = -1;
                for (int dy = p->dy_min; dy <= p->dy_max; ++dy)
                    for (int d = dmin; d <= dmax; ++d) {
                        int c = (dy - p->dy_min) * nd + (d - dmin);
                        Sf[c] = cost_forward(CL, CR, Ws, Hs, px, py, np, d, dy);
                        if (best < 0 || Sf[c] < Sf[best]) best = c;
                    }
                int dy_f = p->dy_min + best / nd, d_f = dmin + best % nd;
                o->d_f = d_f;
                o->dy_f = dy_f;
                o->s_0 = Sf[best];
                o->s_m = d_f > dmin ? Sf[best - 1] : 0;
                o->s_p = d_f < dmax ? Sf[best + 1] : 0;

                /* Backward search from the matched positions (Sec. 4.3.3). */
                int bestb = -1;
                for (int dy = p->dy_min; dy <= p->dy_max; ++dy)
                    for (int d = dmin; d <= dmax; ++d) {
                        int c = (dy - p->dy_min) * nd + (d - dmin);
                        Sb[c] = cost_backward(CL, CR, Ws, Hs, px, py, np, d_f, dy_f, d, dy);
                        if (bestb < 0 || Sb[c] < Sb[bestb]) bestb = c;
                    }
                o->dy_b = p->dy_min + bestb / nd;
                o->d_b = dmin + bestb % nd;

                if (cost_f) memcpy(cost_f + ((size_t)i * slots + s) * nc_max, Sf, sizeof(int32_t) * (size_t)nd * ndy);
                if (cost_b) memcpy(cost_b + ((size_t)i * slots + s) * nc_max, Sb, sizeof(int32_t) * (size_t)nd * ndy);

                /* Eq. subpixel; at a range end there is no neighbour on one side and
                 * the integer argmin is kept. */
                if (d_f == dmin || d_f == dmax) {
                    o->d_sub = (float)d_f;
                    o->flags |= ORC_BLK_SUBPIX_CLAMPED;
                } else {
                    o->d_sub = orc_subpixel(d_f, o->s_m, o->s_0, o->s_p);
                }
                /* Scaled-grid disparity back to full resolution, d_full = k d (Sec. 4.1's rescale). */
                o->d_full = o->d_sub * (float)k;

                /* Consistency: accept iff |dx_v| <= fb_tol with dx_v = d_b - d_f. */
                int dxv = o->d_b - d_f;
                if (dxv < 0) dxv = -dxv;
                if (dxv <= p->fb_tol) {
                    o->flags |= ORC_BLK_VALID;
                    if (o->flags & ORC_BLK_SUBPIX_CLAMPED) clamp_any = 1;
                } else {
                    o->flags |= ORC_BLK_FB_REJECT;
                    fb_any = 1;
                }
            }

            if (fb_any) fl |= ORC_BOX_FB_REJECT;
            if (few_any) fl |= ORC_BOX_FEW_POINTS;
            if (clamp_any) fl |= ORC_BOX_SUBPIX_CLAMPED;

            /* FAR: the box's single block.  CLOSE: robust aggregation. */
            int have = 0;
            float d_box = 0.0f;
            if (far) {
                if (bres[0].flags & ORC_BLK_VALID) { have = 1; d_box = bres[0].d_full; }
            } else {
                int nv = 0;
                for (int s = 0; s < g * g; ++s)
                    if (bres[s].flags & ORC_BLK_VALID) dvals[nv++] = bres[s].d_full;
                have = orc_aggregate(dvals, nv, p->agg_tau_d, p->agg_nmin, p->agg_mode,
                                     p->trim_frac, &d_box);
                if (!have) fl |= ORC_BOX_NO_SEGMENT;
            }
            if (have) {
                if (d_box > 0.0f) {
                    fl |= ORC_BOX_VALID;
                    disp[i] = d_box;
                    depth[i] = orc_depth(f_px, baseline_m, d_box);
                } else {
                    fl |= ORC_BOX_NONPOS_DISP;
                }
            }
            flags[i] = fl;
            if (blk) memcpy(blk + (size_t)i * slots, bres, sizeof(orc_block) * (size_t)(g * g));
        }
    }

    free(CL1); free(CR1); free(CLk); free(CRk);
    free(cb); free(is_far); free(px); free(py); free(Sf); free(Sb); free(occ);
    free(bres); free(dvals);
    return 0;
}

/* Sec. 4.3.6 (Q reprojection, transform to the vehicle frame) and the
 * covariance estimation equation, written out in double. */
void orc_box_points(const int32_t *boxes, const float *disp, const uint8_t *flags, int n,
                    const orc_geometry *geo, int n_geo, double *out)
{
    for (int i = 0; i < n; ++i) {
        double *o = out + 8 * (size_t)i;
        for (int k = 0; k < 8; ++k) o[k] = NAN;
        const int32_t *b = boxes + 5 * (size_t)i;
        const int fi = b[4];
        if (fi < 0 || fi >= n_geo || !(flags[i] & ORC_BOX_VALID)) continue;
        const orc_geometry *g = geo + fi;
        const int x0 = b[0] > 0 ? b[0] : 0, y0 = b[1] > 0 ? b[1] : 0;
        const int x1 = b[2] < g->width ? b[2] : g->width, y1 = b[3] < g->height ? b[3] : g->height;
        if (x1 <= x0 || y1 <= y0) continue;
        const double in[4] = {(x0 + x1 - 1) / 2.0, (y0 + y1 - 1) / 2.0, (double)disp[i], 1.0};
        double h[4];
        for (int r = 0; r < 4; ++r) {
            h[r] = 0.0;
            for (int c = 0; c < 4; ++c) h[r] += g->Q[4 * r + c] * in[c];
        }
        if (h[3] == 0.0) continue;
        const double p[3] = {h[0] / h[3], h[1] / h[3], h[2] / h[3]};
        double pv[3];
        for (int r = 0; r < 3; ++r)
            pv[r] = g->T[4 * r] * p[0] + g->T[4 * r + 1] * p[1] + g->T[4 * r + 2] * p[2] + g->T[4 * r + 3];
        const double Z = p[2];
        const double fb = g->f_px * g->baseline_m;
        o[0] = p[0];
        o[1] = p[1];
        o[2] = p[2];
        o[3] = pv[0];
        o[4] = pv[1];
        o[5] = pv[2];
        o[6] = Z * Z * Z * Z * g->disp_var / (fb * fb);
        o[7] = h[3];
    }
}

/* Sec. 5.1: vertical offset search, census matching per ROI pixel. */
int orc_auto_rect(const uint8_t *L, const uint8_t *R, int W, int H, int pitch, int win_w, int win_h,
                  int sentinel, int rx0, int ry0, int rx1, int ry1, int dmin, int dmax, int delta_min,
                  int delta_max, int d_thresh, int fb_tol, int64_t *counts)
{
    if (dmin > dmax || delta_min > delta_max || rx0 >= rx1 || ry0 >= ry1) return delta_min;
    uint64_t *CL = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * H);
    uint64_t *CR = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W * H);
    orc_census(L, W, H, pitch, 1, win_w, win_h, sentinel, CL);
    orc_census(R, W, H, pitch, 1, win_w, win_h, sentinel, CR);
    int best = delta_min;
    int64_t best_count = -1;
    for (int delta = delta_min; delta <= delta_max; ++delta) {
        int64_t count = 0;
        for (int y = ry0; y < ry1; ++y) {
            for (int x = rx0; x < rx1; ++x) {
                const int yl = y + delta;
                if (x - win_w / 2 < 0 || x + win_w / 2 >= W || yl - win_h / 2 < 0 || yl + win_h / 2 >= H)
                    continue; /* left census undefined */
                const uint64_t cl = code_at(CL, W, H, x, yl);
                int d_f = dmin, s_best = 1 << 30;
                for (int d = dmin; d <= dmax; ++d) {
                    const int s_d = popc64(cl ^ code_at(CR, W, H, x - d, y));
                    if (s_d < s_best) { s_best = s_d; d_f = d; }
                }
                const uint64_t cq = code_at(CR, W, H, x - d_f, y);
                int d_b = dmin;
                s_best = 1 << 30;
                for (int d = dmin; d <= dmax; ++d) {
                    const int s_d = popc64(cq ^ code_at(CL, W, H, x - d_f + d, y + delta));
                    if (s_d < s_best) { s_best = s_d; d_b = d; }
                }
                const int dx = d_b > d_f ? d_b - d_f : d_f - d_b;
                if (dx <= fb_tol && d_f > d_thresh) ++count;
            }
        }
        counts[delta - delta_min] = count;
        if (count > best_count) { best_count = count; best = delta; }
    }
    free(CL);
    free(CR);
    return best;
}

/* Sec. 5.1 temporal filter: sliding-window median, clamped step. */
int orc_rect_filter(const int *estimates, int n, int prev, int max_step)
{
    if (n < 1) return prev;
    int *v = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) v[i] = estimates[i];
    for (int i = 1; i < n; ++i) { /* insertion sort ascending */
        const int t = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
        v[j + 1] = t;
    }
    const int med = v[(n - 1) / 2];
    free(v);
    int step = med - prev;
    if (step > max_step) step = max_step;
    if (step < -max_step) step = -max_step;
    return prev + step;
}
