/*
 * tmd_oracle.c -- plain, serial CPU oracle for TPC track-model encoding and
 * decoding (arXiv:2411.02206, Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the test suite, the smoke check and the CPU-baseline leg of the bench
 * load it.  It shares no source, header, table or helper with the CUDA
 * library; both are written independently from the same format definition.
 *
 * What it computes (Sec. 4):
 *   - track-model encoding: each attached cluster after the first of its track
 *     is stored as the residual of its quantised pad/time to the prediction of
 *     the track model, which is updated with the cluster after each step;
 *   - unattached-cluster encoding: per (sector,row) the clusters are sorted by
 *     position (time, then pad) and stored as differences to the preceding one;
 *   - track-model decoding: the exact inverse of both, producing the native
 *     cluster list grouped by (sector,row), attached clusters first in
 *     (track, cluster) order, then the unattached clusters in stored order;
 *   - entropy coding of the compressed frame's streams (rANS, Sec. 1, 3 and 4; the
 *     format is this project's own, defined with the code below);
 *   - the global (x, y, z) positions of a native list with the nominal
 *     geometry (the decoded clusters feed the downstream tracking).
 *
 * The paper does not give the track model (it is in the cited CTD2019
 * proceedings, not available here).  The model below is this project's
 * reading: a linear Kalman filter in the sector-local frame, with a parabola
 * (y, dy/dx, d2y/dx2) for the bending plane and a line (t, dt/dx) for drift
 * time.  Every floating-point operation is binary32, round-to-nearest-even,
 * performed in the order written; the model's multiply-adds are written as
 * explicit fmaf calls (one rounding each, C99 7.12.13), and this file must be
 * compiled with -ffp-contract=off so that the compiler fuses nothing else.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define O_NSEC 36
#define O_NROW 152
#define O_NBIN (O_NSEC * O_NROW)

/* status bits of a decoded frame */
#define O_ST_COUNT 1u   /* counts inconsistent: sum of nCl, nCl == 0, sum of nUnatt */
#define O_ST_ROW 2u     /* a row >= 152 or a sector >= 36 */
#define O_ST_TIME 4u    /* a decoded time >= 2^24 (does not fit the native record) */

/* ------------------------------------------------------------------------ */
/* Geometry of the synthetic TPC.                                           */
/* Row r lies on the plane x = 85 + r cm of its sector's local frame; it    */
/* holds nPads(r) = 66 + floor(72 r / 151) pads spanning +-x tan(10 deg).   */
/* Sector s (0..17 on the A side, 18..35 on the C side) is centred at the   */
/* azimuth (s mod 18) * 20 deg + 10 deg.                                   */
/* ------------------------------------------------------------------------ */
static float g_x[O_NROW];      /* row plane x [cm] */
static float g_w[O_NROW];      /* pad width [cm] */
static float g_invw[O_NROW];   /* 1 / pad width */
static float g_halfnp[O_NROW]; /* nPads / 2 */
static int g_np[O_NROW];
static float g_cos[18], g_sin[18]; /* cos, sin of k * 20 deg */
static float g_ccen[18], g_scen[18]; /* cos, sin of the sector centres (20 k + 10) deg */
static int g_geo_ready = 0;

/* exact sin/cos of an integer number of degrees by reduction to a reference
 * angle in [0, 90], so that multiples of 90 deg give exact zeros and ones */
static void o_sincos_deg(int a, double* s, double* c) {
  int q = ((a % 360) + 360) % 360;
  double ss = 1.0, sc = 1.0;
  if (q > 180) { q = 360 - q; ss = -1.0; }
  if (q > 90) { q = 180 - q; sc = -1.0; }
  double r = (double)q * (3.14159265358979323846 / 180.0);
  *s = ss * (q == 0 ? 0.0 : (q == 90 ? 1.0 : sin(r)));
  *c = sc * (q == 0 ? 1.0 : (q == 90 ? 0.0 : cos(r)));
}

static void o_geo_init(void) {
  if (g_geo_ready) return;
  const float tan10 = 0.17632698f; /* binary32 nearest tan(10 deg) */
  for (int r = 0; r < O_NROW; r++) {
    int np = 66 + (72 * r) / 151;
    float x = 85.0f + (float)r;
    float w = (2.0f * x * tan10) / (float)np;
    g_np[r] = np;
    g_x[r] = x;
    g_w[r] = w;
    g_invw[r] = 1.0f / w;
    g_halfnp[r] = 0.5f * (float)np;
  }
  for (int k = 0; k < 18; k++) {
    double s, c;
    o_sincos_deg(20 * k, &s, &c);
    g_cos[k] = (float)c;
    g_sin[k] = (float)s;
    o_sincos_deg(20 * k + 10, &s, &c);
    g_ccen[k] = (float)c;
    g_scen[k] = (float)s;
  }
  g_geo_ready = 1;
}

/* ------------------------------------------------------------------------ */
/* Track model parameters.                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  float sy2;  /* measurement variance of y [cm^2] */
  float st2;  /* measurement variance of t [bin^2] */
  float qty;  /* process noise of dy/dx per cm of |dx| */
  float qtt;  /* process noise of dt/dx per cm of |dx| */
  float cty0; /* seed variance of dy/dx */
  float cc0;  /* seed variance of d2y/dx2 [cm^-2] */
  float ctt0; /* seed variance of dt/dx [bin^2/cm^2] */
  float syr;  /* variance of y after a sector or leg change [cm^2] */
  float kc;   /* |d2y/dx2| per unit q/pT [cm^-1 per (GeV/c)^-1] */
} OModel;

static const OModel O_DEFAULT_MODEL = {0.01f, 0.04f, 1.0e-6f, 4.0e-6f, 0.01f,
                                       1.0e-8f, 4.0f, 0.25f, 0.0015f};

/* Track state: sector-local frame, reference plane x. */
typedef struct {
  float x;
  float y, ty, c;               /* y-block: parabola */
  float c00, c01, c02, c11, c12, c22; /* y-block covariance (upper triangle) */
  float t, tt;                  /* t-block: line in drift time */
  float d00, d01, d11;          /* t-block covariance */
  int raw_row;                  /* row walk: header row + row differences, mod 256 */
  int row, sec;                 /* row used by the model: min(raw_row, 151) */
} OState;

/* Quantisation: clamp to [lo, hi] (a NaN goes to lo), then floor(v + 0.5). */
static uint32_t o_quant(float v, float lo, float hi) {
  if (!(v >= lo)) v = lo;
  if (v > hi) v = hi;
  return (uint32_t)floorf(v + 0.5f);
}
#define O_PAD_HI 65535.0f
#define O_TIME_HI 8388607.0f

/* pad code (1/64 pad) -> y [cm] on row r */
static float o_pad_to_y(uint32_t padq, int r) {
  return fmaf((float)padq, 0.015625f, -g_halfnp[r]) * g_w[r];
}
/* time code (1/32 bin) -> t [bin] */
static float o_time_to_t(uint32_t timeq) { return (float)timeq * 0.03125f; }

/* q/pT code -> q/pT [(GeV/c)^-1] */
static float o_qpt(uint8_t qpta) { return ((float)qpta - 127.5f) * 0.078125f; }

/* Seed from the first cluster of the track (stored absolute in the header). */
static void o_seed(const OModel* m, OState* s, uint8_t qpta, int raw_row, int sec,
                   uint32_t padq, uint32_t timeq) {
  float qpt = o_qpt(qpta);
  int row = raw_row < O_NROW ? raw_row : O_NROW - 1;
  s->raw_row = raw_row;
  s->row = row;
  s->sec = sec;
  s->x = g_x[row];
  s->y = o_pad_to_y(padq, row);
  s->c = (-m->kc) * qpt;
  /* slope of the parabola through the origin and the first cluster */
  s->ty = s->y / s->x + (s->c * s->x) * 0.5f;
  s->c00 = m->sy2; s->c01 = 0.0f; s->c02 = 0.0f;
  s->c11 = m->cty0; s->c12 = 0.0f; s->c22 = m->cc0;
  s->t = o_time_to_t(timeq);
  s->tt = 0.0f;
  s->d00 = m->st2; s->d01 = 0.0f; s->d11 = m->ctt0;
}

static void o_reset_ycov(const OModel* m, OState* s) {
  s->c00 = m->syr; s->c01 = 0.0f; s->c02 = 0.0f;
  s->c11 = m->cty0; s->c12 = 0.0f; s->c22 = m->cc0;
}

/* A new leg: the track turns back in x.  The x-parametrised slope and
 * curvature change sign, as does dt/dx; the y-block restarts its uncertainty. */
static void o_leg_change(const OModel* m, OState* s) {
  s->ty = -s->ty;
  s->c = -s->c;
  s->tt = -s->tt;
  s->d01 = -s->d01;
  o_reset_ycov(m, s);
}

/* Move the state into the frame of sector nsec: rotate the point, slope and
 * curvature of the parabola by k * 20 deg; crossing to the other side of the
 * central membrane reverses dt/dx. */
static void o_sector_change(const OModel* m, OState* s, int nsec) {
  int k = ((nsec % 18) - (s->sec % 18) + 18) % 18;
  float ca = g_cos[k], sa = g_sin[k];
  float a = ca + s->ty * sa;
  float b = s->ty * ca - sa;
  if (!(a >= 1.0e-3f || a <= -1.0e-3f)) a = (a < 0.0f) ? -1.0e-3f : 1.0e-3f;
  float nx = s->x * ca + s->y * sa;
  float ny = s->y * ca - s->x * sa;
  float ia = 1.0f / a;
  s->ty = b * ia;
  s->c = s->c * ((ia * ia) * ia);
  s->x = nx;
  s->y = ny;
  if ((s->sec < 18) != (nsec < 18)) {
    s->tt = -s->tt;
    s->d01 = -s->d01;
  }
  s->sec = nsec;
  o_reset_ycov(m, s);
}

/* Propagate the state to the plane of row r (linear model, F = [[1,dx,dx^2/2],
 * [0,1,dx],[0,0,1]] for the y-block and [[1,dx],[0,1]] for the t-block). */
static void o_propagate(const OModel* m, OState* s, int r) {
  float dx = g_x[r] - s->x;
  float adx = fabsf(dx);
  float h = (0.5f * s->c) * dx;
  s->y = fmaf(dx, s->ty + h, s->y);
  s->ty = fmaf(s->c, dx, s->ty);
  s->t = fmaf(s->tt, dx, s->t);
  s->x = g_x[r];
  s->row = r;
  /* y-block: C' = F C F^T + diag(0, qty |dx|, 0) */
  float h2 = (0.5f * dx) * dx;
  float a0 = fmaf(h2, s->c02, fmaf(dx, s->c01, s->c00));
  float a1 = fmaf(h2, s->c12, fmaf(dx, s->c11, s->c01));
  float a2 = fmaf(h2, s->c22, fmaf(dx, s->c12, s->c02));
  float b1 = fmaf(dx, s->c12, s->c11);
  float b2 = fmaf(dx, s->c22, s->c12);
  s->c00 = fmaf(h2, a2, fmaf(dx, a1, a0));
  s->c01 = fmaf(dx, a2, a1);
  s->c02 = a2;
  s->c11 = fmaf(m->qty, adx, fmaf(dx, b2, b1));
  s->c12 = b2;
  /* c22 unchanged */
  /* t-block: D' = G D G^T + diag(0, qtt |dx|) */
  float e0 = fmaf(dx, s->d01, s->d00);
  float e1 = fmaf(dx, s->d11, s->d01);
  s->d00 = fmaf(dx, e1, e0);
  s->d01 = e1;
  s->d11 = fmaf(m->qtt, adx, s->d11);
}

/* Kalman update of both blocks with a measured (y, t). */
static void o_update(const OModel* m, OState* s, float ym, float tm) {
  float inv = 1.0f / (s->c00 + m->sy2);
  float k0 = s->c00 * inv, k1 = s->c01 * inv, k2 = s->c02 * inv;
  float r = ym - s->y;
  s->y = fmaf(k0, r, s->y);
  s->ty = fmaf(k1, r, s->ty);
  s->c = fmaf(k2, r, s->c);
  float c00 = s->c00, c01 = s->c01, c02 = s->c02;
  s->c00 = fmaf(-k0, c00, c00);
  s->c01 = fmaf(-k0, c01, c01);
  s->c02 = fmaf(-k0, c02, c02);
  s->c11 = fmaf(-k1, c01, s->c11);
  s->c12 = fmaf(-k1, c02, s->c12);
  s->c22 = fmaf(-k2, c02, s->c22);
  float invt = 1.0f / (s->d00 + m->st2);
  float g0 = s->d00 * invt, g1 = s->d01 * invt;
  float rt = tm - s->t;
  s->t = fmaf(g0, rt, s->t);
  s->tt = fmaf(g1, rt, s->tt);
  float d00 = s->d00, d01 = s->d01;
  s->d00 = fmaf(-g0, d00, d00);
  s->d01 = fmaf(-g0, d01, d01);
  s->d11 = fmaf(-g1, d01, s->d11);
}

/* Apply the key step (row difference, sector/leg difference) of one cluster,
 * propagate to its row and return the quantised prediction.  Returns 0, or
 * O_ST_ROW if the row left the detector (it is then clamped to 151). */
static uint32_t o_step_predict(const OModel* m, OState* s, uint8_t row_diff,
                               uint8_t slice_leg_diff, uint32_t* pred_padq,
                               uint32_t* pred_timeq, float* pred_y, float* pred_t) {
  uint32_t st = 0;
  int leg = slice_leg_diff / O_NSEC;
  int sd = slice_leg_diff % O_NSEC;
  s->raw_row = (s->raw_row + row_diff) & 255;
  int row = s->raw_row;
  if (row >= O_NROW) { st |= O_ST_ROW; row = O_NROW - 1; }
  if (leg != 0) o_leg_change(m, s);
  if (sd != 0) o_sector_change(m, s, (s->sec + sd) % O_NSEC);
  o_propagate(m, s, row);
  float pp = fmaf(s->y, g_invw[row], g_halfnp[row]);
  *pred_padq = o_quant(pp * 64.0f, 0.0f, O_PAD_HI);
  *pred_timeq = o_quant(s->t * 32.0f, 0.0f, O_TIME_HI);
  if (pred_y) *pred_y = s->y;
  if (pred_t) *pred_t = s->t;
  return st;
}

/* ------------------------------------------------------------------------ */
/* Compressed frame (entropy-decoded CTF) and native output.               */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_tracks, n_attached, n_unattached;
  /* per track: the first cluster stored absolute, plus q/pT and length */
  const uint8_t* qpt;
  const uint8_t* row;
  const uint8_t* slice;
  const uint16_t* pad;
  const uint32_t* time;
  const uint16_t* ncl;
  /* per attached cluster, track order (n_attached entries) */
  const uint16_t* qtot_a;
  const uint16_t* qmax_a;
  const uint8_t* flags_a;
  const uint8_t* sigma_pad_a;
  const uint8_t* sigma_time_a;
  /* per attached cluster after the first of its track (n_attached - n_tracks) */
  const uint8_t* row_diff;
  const uint8_t* slice_leg_diff;
  const uint16_t* pad_res;
  const uint32_t* time_res;
  /* per (sector,row) bin, bin = sector * 152 + row */
  const uint32_t* n_unatt;
  /* per unattached cluster, bin order then stored order */
  const uint16_t* pad_diff_u;
  const uint32_t* time_diff_u;
  const uint16_t* qtot_u;
  const uint16_t* qmax_u;
  const uint8_t* flags_u;
  const uint8_t* sigma_pad_u;
  const uint8_t* sigma_time_u;
} OFrame;

/* Native record, 12 bytes little-endian:
 *   u32 time (low 24 bits) | flags << 24;  u16 pad;  u8 sigmaTime;  u8 sigmaPad;
 *   u16 qMax;  u16 qTot. */
static void o_put_record(uint8_t* dst, uint32_t timeq, uint8_t flags, uint16_t padq,
                         uint8_t sig_time, uint8_t sig_pad, uint16_t qmax, uint16_t qtot) {
  uint32_t w0 = (timeq & 0xFFFFFFu) | ((uint32_t)flags << 24);
  dst[0] = (uint8_t)w0; dst[1] = (uint8_t)(w0 >> 8);
  dst[2] = (uint8_t)(w0 >> 16); dst[3] = (uint8_t)(w0 >> 24);
  dst[4] = (uint8_t)padq; dst[5] = (uint8_t)(padq >> 8);
  dst[6] = sig_time; dst[7] = sig_pad;
  dst[8] = (uint8_t)qmax; dst[9] = (uint8_t)(qmax >> 8);
  dst[10] = (uint8_t)qtot; dst[11] = (uint8_t)(qtot >> 8);
}

/* Walk the keys (row, sector) of every attached cluster, track by track.
 * bins[j] receives sector * 152 + row of cluster j.  Returns status bits. */
static uint32_t o_attached_bins(const OFrame* f, const uint32_t* tstart, uint16_t* bins) {
  uint32_t st = 0;
  for (uint32_t t = 0; t < f->n_tracks; t++) {
    uint32_t j0 = tstart[t], n = f->ncl[t];
    int raw = f->row[t], sec = f->slice[t];
    int row = raw;
    if (row >= O_NROW) { st |= O_ST_ROW; row = O_NROW - 1; }
    if (sec >= O_NSEC) { st |= O_ST_ROW; sec = O_NSEC - 1; }
    bins[j0] = (uint16_t)(sec * O_NROW + row);
    for (uint32_t k = 1; k < n; k++) {
      uint32_t d = j0 - t + k - 1;
      raw = (raw + f->row_diff[d]) & 255;
      row = raw;
      if (row >= O_NROW) { st |= O_ST_ROW; row = O_NROW - 1; }
      sec = (sec + f->slice_leg_diff[d] % O_NSEC) % O_NSEC;
      bins[j0 + k] = (uint16_t)(sec * O_NROW + row);
    }
  }
  return st;
}

/* Decode one frame.
 * native:    (n_attached + n_unattached) * 12 bytes
 * row_start: 5473 entries; row_start[b] is the first record of bin b
 * att_count: 5472 entries (may be NULL); attached records of bin b
 * status:    out, O_ST_* bits.  On O_ST_COUNT nothing else is written.
 * Returns 0, or -1 on allocation failure. */
int tmd_oracle_decode(const OFrame* f, uint8_t* native, uint32_t* row_start,
                      uint32_t* att_count, uint32_t* status) {
  o_geo_init();
  const OModel* m = &O_DEFAULT_MODEL;
  uint32_t st = 0;
  /* counts */
  uint64_t sum = 0;
  for (uint32_t t = 0; t < f->n_tracks; t++) {
    if (f->ncl[t] == 0) st |= O_ST_COUNT;
    sum += f->ncl[t];
  }
  if (sum != f->n_attached) st |= O_ST_COUNT;
  uint64_t sumu = 0;
  for (int b = 0; b < O_NBIN; b++) sumu += f->n_unatt[b];
  if (sumu != f->n_unattached) st |= O_ST_COUNT;
  if (st & O_ST_COUNT) { *status = st; return 0; }

  uint32_t* tstart = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)f->n_tracks + 1));
  uint16_t* bins = (uint16_t*)malloc(sizeof(uint16_t) * ((size_t)f->n_attached + 1));
  uint32_t* cursor = (uint32_t*)malloc(sizeof(uint32_t) * O_NBIN);
  uint32_t* attc = (uint32_t*)calloc(O_NBIN, sizeof(uint32_t));
  if (!tstart || !bins || !cursor || !attc) {
    free(tstart); free(bins); free(cursor); free(attc);
    return -1;
  }
  tstart[0] = 0;
  for (uint32_t t = 0; t < f->n_tracks; t++) tstart[t + 1] = tstart[t] + f->ncl[t];

  /* row offsets: attached count + unattached count per bin, exclusive scan */
  st |= o_attached_bins(f, tstart, bins);
  for (uint32_t j = 0; j < f->n_attached; j++) attc[bins[j]]++;
  uint32_t acc = 0;
  for (int b = 0; b < O_NBIN; b++) {
    row_start[b] = acc;
    cursor[b] = acc;
    acc += attc[b] + f->n_unatt[b];
  }
  row_start[O_NBIN] = acc;
  if (att_count) memcpy(att_count, attc, sizeof(uint32_t) * O_NBIN);

  /* attached clusters: tracks in order, clusters in order */
  for (uint32_t t = 0; t < f->n_tracks; t++) {
    uint32_t j0 = tstart[t], n = f->ncl[t];
    int sec0 = f->slice[t] < O_NSEC ? f->slice[t] : O_NSEC - 1;
    OState s;
    o_seed(m, &s, f->qpt[t], f->row[t], sec0, f->pad[t], f->time[t]);
    uint32_t padq = f->pad[t], timeq = f->time[t];
    for (uint32_t k = 0; k < n; k++) {
      uint32_t j = j0 + k;
      if (k > 0) {
        uint32_t d = j0 - t + k - 1, ppad, ptime;
        st |= o_step_predict(m, &s, f->row_diff[d], f->slice_leg_diff[d], &ppad, &ptime,
                             NULL, NULL);
        padq = (ppad + f->pad_res[d]) & 0xFFFFu;
        timeq = ptime + f->time_res[d];
        o_update(m, &s, o_pad_to_y(padq, s.row), o_time_to_t(timeq));
      }
      if (timeq > 0xFFFFFFu) st |= O_ST_TIME;
      uint32_t b = bins[j];
      o_put_record(native + (size_t)12 * cursor[b]++, timeq, f->flags_a[j], (uint16_t)padq,
                   f->sigma_time_a[j], f->sigma_pad_a[j], f->qmax_a[j], f->qtot_a[j]);
    }
  }

  /* unattached clusters: per bin, running sums of the stored differences */
  uint64_t u = 0;
  for (int b = 0; b < O_NBIN; b++) {
    uint32_t padq = 0, timeq = 0;
    for (uint32_t i = 0; i < f->n_unatt[b]; i++, u++) {
      padq = (padq + f->pad_diff_u[u]) & 0xFFFFu;
      timeq = timeq + f->time_diff_u[u];
      if (timeq > 0xFFFFFFu) st |= O_ST_TIME;
      o_put_record(native + (size_t)12 * cursor[b]++, timeq, f->flags_u[u], (uint16_t)padq,
                   f->sigma_time_u[u], f->sigma_pad_u[u], f->qmax_u[u], f->qtot_u[u]);
    }
  }
  free(tstart); free(bins); free(cursor); free(attc);
  *status = st;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Encoder (the synchronous side of Sec. 4), used to build test frames     */
/* whose decoded result is known: the quantised truth itself.              */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_tracks, n_attached, n_unattached;
  const uint8_t* qpt;  /* per track */
  const uint16_t* ncl; /* per track */
  /* per attached cluster, track order */
  const uint8_t* row;
  const uint8_t* sector;
  const uint8_t* leg; /* leg index along the track, non-decreasing */
  const uint16_t* pad;
  const uint32_t* time;
  const uint16_t* qtot_a;
  const uint16_t* qmax_a;
  const uint8_t* flags_a;
  const uint8_t* sigma_pad_a;
  const uint8_t* sigma_time_a;
  /* unattached clusters, any order */
  const uint8_t* row_u;
  const uint8_t* sector_u;
  const uint16_t* pad_u;
  const uint32_t* time_u;
  const uint16_t* qtot_u;
  const uint16_t* qmax_u;
  const uint8_t* flags_u;
  const uint8_t* sigma_pad_u;
  const uint8_t* sigma_time_u;
} OTruth;

/* Writable compressed frame: same fields as OFrame. */
typedef struct {
  uint8_t* qpt; uint8_t* row; uint8_t* slice; uint16_t* pad; uint32_t* time; uint16_t* ncl;
  uint16_t* qtot_a; uint16_t* qmax_a; uint8_t* flags_a; uint8_t* sigma_pad_a; uint8_t* sigma_time_a;
  uint8_t* row_diff; uint8_t* slice_leg_diff; uint16_t* pad_res; uint32_t* time_res;
  uint32_t* n_unatt;
  uint16_t* pad_diff_u; uint32_t* time_diff_u; uint16_t* qtot_u; uint16_t* qmax_u;
  uint8_t* flags_u; uint8_t* sigma_pad_u; uint8_t* sigma_time_u;
} OFrameOut;

/* unattached sort key: (time, pad), ties by input index (stable) */
static const OTruth* g_sort_truth;
static int o_cmp_unatt(const void* pa, const void* pb) {
  uint32_t a = *(const uint32_t*)pa, b = *(const uint32_t*)pb;
  const OTruth* T = g_sort_truth;
  if (T->time_u[a] != T->time_u[b]) return T->time_u[a] < T->time_u[b] ? -1 : 1;
  if (T->pad_u[a] != T->pad_u[b]) return T->pad_u[a] < T->pad_u[b] ? -1 : 1;
  return a < b ? -1 : (a > b);
}

/* Encode a truth frame.  Returns 0, -1 on allocation failure, -2 on invalid
 * truth (row >= 152, sector >= 36, nCl == 0, inconsistent counts, decreasing
 * leg index). */
int tmd_oracle_encode(const OTruth* T, OFrameOut* o) {
  o_geo_init();
  const OModel* m = &O_DEFAULT_MODEL;
  uint64_t sum = 0;
  for (uint32_t t = 0; t < T->n_tracks; t++) {
    if (T->ncl[t] == 0) return -2;
    sum += T->ncl[t];
  }
  if (sum != T->n_attached) return -2;
  for (uint32_t j = 0; j < T->n_attached; j++)
    if (T->row[j] >= O_NROW || T->sector[j] >= O_NSEC) return -2;
  for (uint32_t i = 0; i < T->n_unattached; i++)
    if (T->row_u[i] >= O_NROW || T->sector_u[i] >= O_NSEC) return -2;

  uint32_t j0 = 0;
  for (uint32_t t = 0; t < T->n_tracks; t++) {
    uint32_t n = T->ncl[t];
    for (uint32_t k = 1; k < n; k++)
      if (T->leg[j0 + k] < T->leg[j0 + k - 1]) return -2;
    o->qpt[t] = T->qpt[t];
    o->row[t] = T->row[j0];
    o->slice[t] = T->sector[j0];
    o->pad[t] = T->pad[j0];
    o->time[t] = T->time[j0];
    o->ncl[t] = (uint16_t)n;
    OState s;
    o_seed(m, &s, T->qpt[t], T->row[j0], T->sector[j0], T->pad[j0], T->time[j0]);
    for (uint32_t k = 1; k < n; k++) {
      uint32_t j = j0 + k, d = j0 - t + k - 1, ppad, ptime;
      int legd = T->leg[j] != T->leg[j - 1] ? 1 : 0;
      int secd = ((int)T->sector[j] - (int)T->sector[j - 1] + O_NSEC) % O_NSEC;
      o->row_diff[d] = (uint8_t)((T->row[j] - T->row[j - 1]) & 255);
      o->slice_leg_diff[d] = (uint8_t)(legd * O_NSEC + secd);
      o_step_predict(m, &s, o->row_diff[d], o->slice_leg_diff[d], &ppad, &ptime, NULL, NULL);
      o->pad_res[d] = (uint16_t)((T->pad[j] - ppad) & 0xFFFFu);
      o->time_res[d] = T->time[j] - ptime;
      o_update(m, &s, o_pad_to_y(T->pad[j], s.row), o_time_to_t(T->time[j]));
    }
    j0 += n;
  }
  if (T->n_attached) { /* (memcpy from or to a null pointer is undefined even for 0 bytes) */
    memcpy(o->qtot_a, T->qtot_a, 2u * T->n_attached);
    memcpy(o->qmax_a, T->qmax_a, 2u * T->n_attached);
    memcpy(o->flags_a, T->flags_a, T->n_attached);
    memcpy(o->sigma_pad_a, T->sigma_pad_a, T->n_attached);
    memcpy(o->sigma_time_a, T->sigma_time_a, T->n_attached);
  }

  /* unattached: group by bin (stable), sort each bin by (time, pad), store
   * differences to the preceding cluster (the first to zero) */
  uint32_t nu = T->n_unattached;
  uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)nu + 1));
  uint32_t* start = (uint32_t*)calloc(O_NBIN + 1, sizeof(uint32_t));
  uint32_t* cur = (uint32_t*)malloc(sizeof(uint32_t) * O_NBIN);
  if (!idx || !start || !cur) { free(idx); free(start); free(cur); return -1; }
  for (uint32_t i = 0; i < nu; i++) start[T->sector_u[i] * O_NROW + T->row_u[i] + 1]++;
  for (int b = 0; b < O_NBIN; b++) {
    o->n_unatt[b] = start[b + 1];
    start[b + 1] += start[b];
    cur[b] = start[b];
  }
  for (uint32_t i = 0; i < nu; i++) idx[cur[T->sector_u[i] * O_NROW + T->row_u[i]]++] = i;
  g_sort_truth = T;
  for (int b = 0; b < O_NBIN; b++)
    qsort(idx + start[b], start[b + 1] - start[b], sizeof(uint32_t), o_cmp_unatt);
  for (int b = 0; b < O_NBIN; b++) {
    uint32_t ppad = 0, ptime = 0;
    for (uint32_t p = start[b]; p < start[b + 1]; p++) {
      uint32_t i = idx[p];
      o->pad_diff_u[p] = (uint16_t)((T->pad_u[i] - ppad) & 0xFFFFu);
      o->time_diff_u[p] = T->time_u[i] - ptime;
      ppad = T->pad_u[i];
      ptime = T->time_u[i];
      o->qtot_u[p] = T->qtot_u[i];
      o->qmax_u[p] = T->qmax_u[i];
      o->flags_u[p] = T->flags_u[i];
      o->sigma_pad_u[p] = T->sigma_pad_u[i];
      o->sigma_time_u[p] = T->sigma_time_u[i];
    }
  }
  free(idx); free(start); free(cur);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Introspection for the tests that pin the model.                         */
/* ------------------------------------------------------------------------ */

/* Run the track model along one track with known measurements (the encoder's
 * view).  model: 9 floats in OModel order, or NULL for the default model.
 * For every cluster k the arrays receive: pred_y/pred_t the propagated state
 * before the update (k = 0: the seed), pred_padq/pred_timeq the quantised
 * prediction (k = 0: the stored header values), state (17 floats per k) the
 * state after the update: x y ty c c00 c01 c02 c11 c12 c22 t tt d00 d01 d11
 * row sec.  Returns status bits. */
uint32_t tmd_oracle_track_trace(const float* model, uint8_t qpta, uint32_t n,
                                const uint8_t* row, const uint8_t* sector, const uint8_t* leg,
                                const uint16_t* pad, const uint32_t* time, float* pred_y,
                                float* pred_t, uint32_t* pred_padq, uint32_t* pred_timeq,
                                float* state) {
  o_geo_init();
  OModel mm = O_DEFAULT_MODEL;
  if (model) memcpy(&mm, model, sizeof(OModel));
  uint32_t st = 0;
  OState s;
  if (n == 0) return 0;
  o_seed(&mm, &s, qpta, row[0], sector[0], pad[0], time[0]);
  for (uint32_t k = 0; k < n; k++) {
    if (k == 0) {
      pred_y[0] = s.y; pred_t[0] = s.t;
      pred_padq[0] = pad[0]; pred_timeq[0] = time[0];
    } else {
      uint8_t rd = (uint8_t)((row[k] - row[k - 1]) & 255);
      int legd = leg[k] != leg[k - 1] ? 1 : 0;
      int secd = ((int)sector[k] - (int)sector[k - 1] + O_NSEC) % O_NSEC;
      st |= o_step_predict(&mm, &s, rd, (uint8_t)(legd * O_NSEC + secd), &pred_padq[k],
                           &pred_timeq[k], &pred_y[k], &pred_t[k]);
      o_update(&mm, &s, o_pad_to_y(pad[k], s.row), o_time_to_t(time[k]));
    }
    float* o = state + 17 * (size_t)k;
    o[0] = s.x; o[1] = s.y; o[2] = s.ty; o[3] = s.c;
    o[4] = s.c00; o[5] = s.c01; o[6] = s.c02; o[7] = s.c11; o[8] = s.c12; o[9] = s.c22;
    o[10] = s.t; o[11] = s.tt; o[12] = s.d00; o[13] = s.d01; o[14] = s.d11;
    o[15] = (float)s.row; o[16] = (float)s.sec;
  }
  return st;
}

/* Apply one sector change to a given state (x, y, ty, c) and report the
 * rotated (x, y, ty, c). */
void tmd_oracle_rotate(int from_sec, int to_sec, const float* in4, float* out4) {
  o_geo_init();
  OState s;
  memset(&s, 0, sizeof(s));
  s.x = in4[0]; s.y = in4[1]; s.ty = in4[2]; s.c = in4[3]; s.sec = from_sec;
  o_sector_change(&O_DEFAULT_MODEL, &s, to_sec);
  out4[0] = s.x; out4[1] = s.y; out4[2] = s.ty; out4[3] = s.c;
}

uint32_t tmd_oracle_quant(float v, float lo, float hi) { return o_quant(v, lo, hi); }

/* Geometry tables: x[152], w[152], invw[152], np[152], cos[18], sin[18]. */
void tmd_oracle_geometry(float* x, float* w, float* invw, int32_t* np, float* cs, float* sn) {
  o_geo_init();
  for (int r = 0; r < O_NROW; r++) { x[r] = g_x[r]; w[r] = g_w[r]; invw[r] = g_invw[r]; np[r] = g_np[r]; }
  for (int k = 0; k < 18; k++) { cs[k] = g_cos[k]; sn[k] = g_sin[k]; }
}

/* Sector-centre tables: cos, sin of (20 k + 10) deg, k = 0..17. */
void tmd_oracle_sector_centres(float* cs, float* sn) {
  o_geo_init();
  for (int k = 0; k < 18; k++) { cs[k] = g_ccen[k]; sn[k] = g_scen[k]; }
}

/* ------------------------------------------------------------------------ */
/* Global positions of the clusters of a native list, with the nominal     */
/* geometry of the synthetic TPC (the decoded clusters feed the tracking of */
/* the asynchronous chain, Sec. 1 and 3; real calibration maps are not          */
/* available).  Record i of bin (s, r) (row_start[b] <= i < row_start[b+1]) */
/* with pad code P and time code T:                                         */
/*   local  x = 85 + r, y = (P/64 - nPads(r)/2) * w(r)  (the model's pad_to_y) */
/*   global X = x cos(psi) - y sin(psi), Y = x sin(psi) + y cos(psi),       */
/*          psi = (s mod 18) * 20 + 10 deg (the sector centre)              */
/*   drift  |Z| = 250 - 0.5 * (T / 32), positive for sectors 0-17.          */
/* binary32, in the order written (the pad term is one fmaf).               */
/* ------------------------------------------------------------------------ */
void tmd_oracle_global_xyz(const uint8_t* native, const uint32_t* row_start, uint32_t n,
                           float* gx, float* gy, float* gz) {
  o_geo_init();
  for (int b = 0; b < O_NBIN; b++) {
    const int s = b / O_NROW, r = b % O_NROW;
    const float ca = g_ccen[s % 18], sa = g_scen[s % 18];
    for (uint32_t i = row_start[b]; i < row_start[b + 1] && i < n; i++) {
      const uint8_t* rec = native + (size_t)i * 12;
      const uint32_t tcode = (uint32_t)rec[0] | ((uint32_t)rec[1] << 8) | ((uint32_t)rec[2] << 16);
      const uint32_t pcode = (uint32_t)rec[4] | ((uint32_t)rec[5] << 8);
      const float yl = o_pad_to_y(pcode, r);
      const float t = (float)tcode * 0.03125f;
      const float zabs = 250.0f - t * 0.5f;
      gx[i] = g_x[r] * ca - yl * sa;
      gy[i] = g_x[r] * sa + yl * ca;
      gz[i] = s < 18 ? zabs : -zabs;
    }
  }
}

/* Default model parameters (9 floats, OModel order). */
void tmd_oracle_default_model(float* out9) { memcpy(out9, &O_DEFAULT_MODEL, sizeof(OModel)); }

/* ------------------------------------------------------------------------ */
/* Entropy coding of a compressed frame: the step before track-model        */
/* decoding (Sec. 1, 3 and 4: the CTF's streams are entropy coded with rANS, and   */
/* the entropy decoding feeds the track-model decoding).  The ALICE rANS    */
/* format is not available; this is the project's own format, written from  */
/* the definition of range asymmetric numeral systems (rANS, J. Duda,       */
/* arXiv:1311.2540):                                                        */
/*   scale M = 2^12.  Symbol s has frequency f_s (sum of all f = M) and     */
/*   cumulative frequency c_s = sum of f_t over t < s; it owns the slots    */
/*   [c_s, c_s + f_s) of [0, M).                                            */
/*   encode s:  x -> (x div f_s) * M + c_s + (x mod f_s)                    */
/*   decode:    slot = x mod M, s = the symbol owning slot,                 */
/*              x -> f_s * (x div M) + slot - c_s                           */
/*   The state stays in [2^16, 2^32): before s is encoded, while            */
/*   x >= f_s * 2^20 the low 16 bits are emitted as a word and x >>= 16;    */
/*   after a symbol is decoded, while x < 2^16, x = (x << 16) | next word.  */
/*   A stream starts (encoder) and ends (decoder) at x = 2^16.              */
/*                                                                          */
/* Symbols are the bytes of the values: a field of width w (1, 2, 4 bytes)  */
/* has w byte planes, each with its own 256-entry frequency table; value i  */
/* is coded as its bytes, least significant first.  A field of n values is   */
/* cut into chunks of 32 * 256 values; lane l (0..31) of a chunk codes the  */
/* values 32 k + l (k = 0..255) of the chunk, each lane its own rANS stream. */
/*                                                                          */
/* Frequency normalisation (count n_s of symbol s among the n bytes of a     */
/* plane): f_s = 0 if n_s = 0, else max(1, floor(n_s * M / n)); then a      */
/* deficit M - sum f is added to the symbol with the largest count (lowest  */
/* symbol on ties), and while the sum exceeds M, 1 is taken from the symbol  */
/* with the largest f (lowest symbol on ties).  n = 0: f_0 = M.             */
/*                                                                          */
/* Byte layout (little-endian; every offset a multiple of 16):              */
/*   frame header, 32 bytes: u32 magic 0x52444D54 ("TMDR"), version 1,      */
/*     number of fields 23, values per lane per chunk 256, n_tracks,        */
/*     n_attached, n_unattached, 0;                                         */
/*   23 directory entries of 32 bytes, fields in the order of the frame     */
/*     streams (qpt .. sigma_time_u): u64 section offset from the start,    */
/*     u64 section bytes, u32 n, u32 width, u32 chunks, u32 0;              */
/*   field section: u16 freq[w][256]; u32 state[chunks][32] (each lane's    */
/*     decoder start state); u32 woff[chunks + 1] (chunk c's words occupy   */
/*     u32 slots [woff[c], woff[c+1]) of the word area, a multiple of 32);  */
/*     zero padding to 16 bytes; the word area: slot woff[c] + 32 j + l     */
/*     holds lane l's words 2j (low half) and 2j + 1 (high half) in         */
/*     decoding order, zero past the lane's last word.                      */
/* ------------------------------------------------------------------------ */
#define O_R_M 4096u
#define O_R_LOWER 65536u
#define O_R_K 256u
#define O_R_CHUNK (32u * O_R_K)
#define O_R_MAGIC 0x52444D54u
#define O_R_NFIELD 23
#define O_R_HEAD (32u + 32u * O_R_NFIELD)
#define O_R_CORRUPT (-4)

static void o_put16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void o_put32(uint8_t* p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void o_put64(uint8_t* p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint32_t o_get16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t o_get32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint64_t o_get64(const uint8_t* p) {
  return (uint64_t)o_get32(p) | ((uint64_t)o_get32(p + 4) << 32);
}
static uint64_t o_align16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

/* value i of a field of width w, and its byte p */
static uint32_t o_value(const void* a, uint32_t w, uint32_t i) {
  if (w == 1) return ((const uint8_t*)a)[i];
  if (w == 2) return ((const uint16_t*)a)[i];
  return ((const uint32_t*)a)[i];
}
static void o_set_value(void* a, uint32_t w, uint32_t i, uint32_t v) {
  if (w == 1) ((uint8_t*)a)[i] = (uint8_t)v;
  else if (w == 2) ((uint16_t*)a)[i] = (uint16_t)v;
  else ((uint32_t*)a)[i] = v;
}

static void o_rans_normalise(const uint64_t* count, uint64_t n, uint32_t* f) {
  if (n == 0) {
    for (int s = 0; s < 256; s++) f[s] = 0;
    f[0] = O_R_M;
    return;
  }
  uint64_t sum = 0;
  int smax = 0;
  for (int s = 0; s < 256; s++) {
    if (count[s] == 0) f[s] = 0;
    else {
      uint64_t v = count[s] * O_R_M / n;
      f[s] = v < 1 ? 1u : (uint32_t)v;
    }
    sum += f[s];
    if (count[s] > count[smax]) smax = s;
  }
  if (sum < O_R_M) f[smax] += (uint32_t)(O_R_M - sum);
  while (sum > O_R_M) {
    int b = -1;
    for (int s = 0; s < 256; s++)
      if (f[s] > 1 && (b < 0 || f[s] > f[b])) b = s;
    f[b] -= 1;
    sum -= 1;
  }
}

/* Fixed part of a field section: freq tables, states, chunk offsets. */
static uint64_t o_rans_fixed(uint32_t n, uint32_t w) {
  uint64_t nch = ((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK;
  return o_align16(512u * (uint64_t)w + 128u * nch + 4u * (nch + 1));
}

/* Largest possible section: every symbol emits a word. */
uint64_t tmd_oracle_rans_field_bound(uint32_t n, uint32_t w) {
  uint64_t nch = ((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK;
  return o_align16(o_rans_fixed(n, w) + nch * 32u * 4u * ((O_R_K * w + 1) / 2));
}

/* Encode one field (n values of width w) into a section.  Returns 0, -1 on
 * allocation failure, -3 if cap is too small. */
int tmd_oracle_rans_field_encode(const void* vals, uint32_t n, uint32_t w, uint8_t* out,
                                 uint64_t cap, uint64_t* size) {
  const uint32_t nch = (uint32_t)(((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK);
  uint32_t f[4][256], c[4][256];
  for (uint32_t p = 0; p < w; p++) {
    uint64_t count[256] = {0};
    for (uint32_t i = 0; i < n; i++) count[(o_value(vals, w, i) >> (8 * p)) & 0xFFu]++;
    o_rans_normalise(count, n, f[p]);
    uint32_t acc = 0;
    for (int s = 0; s < 256; s++) { c[p][s] = acc; acc += f[p][s]; }
  }
  const uint64_t a_state = 512u * (uint64_t)w, a_woff = a_state + 128u * (uint64_t)nch;
  const uint64_t a_words = o_rans_fixed(n, w);
  if (cap < a_words) return -3;
  memset(out, 0, a_words);
  for (uint32_t p = 0; p < w; p++)
    for (int s = 0; s < 256; s++) o_put16(out + 2 * (256 * p + s), f[p][s]);

  uint16_t* stack = (uint16_t*)malloc(sizeof(uint16_t) * O_R_K * 4);
  uint16_t* words = (uint16_t*)malloc(sizeof(uint16_t) * 32 * (O_R_K * 4 + 1));
  uint32_t nw[32];
  if (!stack || !words) { free(stack); free(words); return -1; }
  uint64_t woff = 0; /* u32 slots used so far */
  for (uint32_t ch = 0; ch < nch; ch++) {
    uint32_t maxpairs = 0;
    for (uint32_t l = 0; l < 32; l++) {
      /* this lane's values, in decoding order: i = base + 32 k + l */
      const uint64_t base = (uint64_t)ch * O_R_CHUNK + l;
      uint32_t nk = 0;
      while (nk < O_R_K && base + 32u * nk < n) nk++;
      uint32_t x = O_R_LOWER, ns = 0;
      /* encode in reverse decoding order: values last to first, bytes high to low */
      for (uint32_t k = nk; k-- > 0;) {
        const uint32_t v = o_value(vals, w, (uint32_t)(base + 32u * k));
        for (uint32_t p = w; p-- > 0;) {
          const uint32_t s = (v >> (8 * p)) & 0xFFu, fs = f[p][s];
          if ((uint64_t)x >= ((uint64_t)fs << 20)) {
            stack[ns++] = (uint16_t)(x & 0xFFFFu);
            x >>= 16;
          }
          x = (x / fs) * O_R_M + c[p][s] + (x % fs);
        }
      }
      o_put32(out + a_state + 4u * (32u * (uint64_t)ch + l), x);
      /* the decoder reads the words in the reverse order of emission */
      for (uint32_t q = 0; q < ns; q++) words[l * (O_R_K * 4 + 1) + q] = stack[ns - 1 - q];
      nw[l] = ns;
      if ((ns + 1) / 2 > maxpairs) maxpairs = (ns + 1) / 2;
    }
    o_put32(out + a_woff + 4u * (uint64_t)ch, (uint32_t)woff);
    const uint64_t need = a_words + 4u * (woff + 32u * (uint64_t)maxpairs);
    if (need > cap) { free(stack); free(words); return -3; }
    for (uint32_t j = 0; j < maxpairs; j++)
      for (uint32_t l = 0; l < 32; l++) {
        const uint32_t q = 2 * j;
        const uint32_t lo = q < nw[l] ? words[l * (O_R_K * 4 + 1) + q] : 0u;
        const uint32_t hi = q + 1 < nw[l] ? words[l * (O_R_K * 4 + 1) + q + 1] : 0u;
        o_put32(out + a_words + 4u * (woff + 32u * j + l), lo | (hi << 16));
      }
    woff += 32u * (uint64_t)maxpairs;
  }
  o_put32(out + a_woff + 4u * (uint64_t)nch, (uint32_t)woff);
  free(stack);
  free(words);
  uint64_t total = o_align16(a_words + 4u * woff);
  if (total > cap) return -3;
  memset(out + a_words + 4u * woff, 0, total - (a_words + 4u * woff));
  *size = total;
  return 0;
}

/* Decode one field section of `bytes` bytes into n values of width w.
 * Returns 0, or -4 if the section is malformed or a stream fails its checks
 * (a lane runs out of words, or does not end at the start state 2^16). */
int tmd_oracle_rans_field_decode(const uint8_t* sec, uint64_t bytes, uint32_t n, uint32_t w,
                                 void* vals) {
  const uint32_t nch = (uint32_t)(((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK);
  const uint64_t a_state = 512u * (uint64_t)w, a_woff = a_state + 128u * (uint64_t)nch;
  const uint64_t a_words = o_rans_fixed(n, w);
  if (w != 1 && w != 2 && w != 4) return O_R_CORRUPT;
  if (bytes < a_words) return O_R_CORRUPT;
  /* the symbol owning each slot, per plane */
  uint32_t f[4][256], c[4][256];
  uint8_t slot_sym[4][O_R_M];
  for (uint32_t p = 0; p < w; p++) {
    uint32_t acc = 0;
    for (int s = 0; s < 256; s++) {
      f[p][s] = o_get16(sec + 2 * (256 * p + s));
      c[p][s] = acc;
      for (uint32_t t = 0; t < f[p][s] && acc + t < O_R_M; t++) slot_sym[p][acc + t] = (uint8_t)s;
      acc += f[p][s];
    }
    if (acc != O_R_M) return O_R_CORRUPT;
  }
  const uint64_t area = (bytes - a_words) / 4u; /* u32 slots available */
  if (o_get32(sec + a_woff) != 0) return O_R_CORRUPT;
  int bad = 0;
  for (uint32_t ch = 0; ch < nch; ch++) {
    const uint64_t w0 = o_get32(sec + a_woff + 4u * (uint64_t)ch);
    const uint64_t w1 = o_get32(sec + a_woff + 4u * ((uint64_t)ch + 1));
    if (w1 < w0 || (w1 - w0) % 32u != 0 || w1 > area) return O_R_CORRUPT;
    const uint32_t maxpairs = (uint32_t)((w1 - w0) / 32u);
    for (uint32_t l = 0; l < 32; l++) {
      const uint64_t base = (uint64_t)ch * O_R_CHUNK + l;
      uint32_t x = o_get32(sec + a_state + 4u * (32u * (uint64_t)ch + l));
      uint32_t q = 0; /* next word of this lane */
      for (uint32_t k = 0; k < O_R_K && base + 32u * k < n; k++) {
        uint32_t v = 0;
        for (uint32_t p = 0; p < w; p++) {
          const uint32_t slot = x % O_R_M, s = slot_sym[p][slot];
          x = f[p][s] * (x / O_R_M) + slot - c[p][s];
          v |= s << (8 * p);
          while (x < O_R_LOWER) {
            uint32_t word = 0;
            if (q / 2 < maxpairs) {
              const uint32_t pair = o_get32(sec + a_words + 4u * (w0 + 32u * (q / 2) + l));
              word = (q % 2) ? pair >> 16 : pair & 0xFFFFu;
            } else {
              bad = 1; /* out of words: the value is garbage, keep going */
            }
            q++;
            x = (x << 16) | word;
            if (x < O_R_LOWER) { bad = 1; break; }
          }
        }
        o_set_value(vals, w, (uint32_t)(base + 32u * k), v);
      }
      if (x != O_R_LOWER) bad = 1;
    }
  }
  return bad ? O_R_CORRUPT : 0;
}

/* Field f (0..22) of a frame: array, width and length. */
static void o_frame_field(const OFrame* F, int i, const void** a, uint32_t* w, uint32_t* n) {
  const uint32_t nt = F->n_tracks, na = F->n_attached, nu = F->n_unattached, nd = na - nt;
  const void* arr[O_R_NFIELD] = {F->qpt, F->row, F->slice, F->pad, F->time, F->ncl,
                                 F->qtot_a, F->qmax_a, F->flags_a, F->sigma_pad_a,
                                 F->sigma_time_a, F->row_diff, F->slice_leg_diff, F->pad_res,
                                 F->time_res, F->n_unatt, F->pad_diff_u, F->time_diff_u,
                                 F->qtot_u, F->qmax_u, F->flags_u, F->sigma_pad_u,
                                 F->sigma_time_u};
  static const uint32_t width[O_R_NFIELD] = {1, 1, 1, 2, 4, 2, 2, 2, 1, 1, 1, 1,
                                             1, 2, 4, 4, 2, 4, 2, 2, 1, 1, 1};
  const uint32_t len[O_R_NFIELD] = {nt, nt, nt, nt, nt, nt, na, na, na, na, na, nd,
                                    nd, nd, nd, O_NBIN, nu, nu, nu, nu, nu, nu, nu};
  *a = arr[i];
  *w = width[i];
  *n = len[i];
}

uint64_t tmd_oracle_rans_frame_bound(const OFrame* F) {
  if (F->n_attached < F->n_tracks) return 0;
  uint64_t total = O_R_HEAD;
  for (int i = 0; i < O_R_NFIELD; i++) {
    const void* a;
    uint32_t w, n;
    o_frame_field(F, i, &a, &w, &n);
    total += tmd_oracle_rans_field_bound(n, w);
  }
  return total;
}

/* Encode a compressed frame (its 23 streams) into one coded frame.  Returns
 * 0, -1 on allocation failure, -2 if n_attached < n_tracks, -3 if cap is too
 * small. */
int tmd_oracle_rans_frame_encode(const OFrame* F, uint8_t* out, uint64_t cap, uint64_t* size) {
  if (F->n_attached < F->n_tracks) return -2;
  if (cap < O_R_HEAD) return -3;
  memset(out, 0, O_R_HEAD);
  o_put32(out, O_R_MAGIC);
  o_put32(out + 4, 1);
  o_put32(out + 8, O_R_NFIELD);
  o_put32(out + 12, O_R_K);
  o_put32(out + 16, F->n_tracks);
  o_put32(out + 20, F->n_attached);
  o_put32(out + 24, F->n_unattached);
  uint64_t off = O_R_HEAD;
  for (int i = 0; i < O_R_NFIELD; i++) {
    const void* a;
    uint32_t w, n;
    o_frame_field(F, i, &a, &w, &n);
    uint64_t used = 0;
    const int rc = tmd_oracle_rans_field_encode(a, n, w, out + off, cap - off, &used);
    if (rc != 0) return rc;
    uint8_t* d = out + 32 + 32 * i;
    o_put64(d, off);
    o_put64(d + 8, used);
    o_put32(d + 16, n);
    o_put32(d + 20, w);
    o_put32(d + 24, (uint32_t)(((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK));
    off += used;
  }
  *size = off;
  return 0;
}

/* Decode a coded frame of `bytes` bytes whose counts must be those of F (the
 * arrays of F are not read); the streams are written to o.  Returns 0 or -4
 * (malformed or failing its stream checks). */
int tmd_oracle_rans_frame_decode(const uint8_t* blob, uint64_t bytes, const OFrame* F,
                                 OFrameOut* o) {
  if (bytes < O_R_HEAD) return O_R_CORRUPT;
  if (o_get32(blob) != O_R_MAGIC || o_get32(blob + 4) != 1 || o_get32(blob + 8) != O_R_NFIELD ||
      o_get32(blob + 12) != O_R_K || o_get32(blob + 16) != F->n_tracks ||
      o_get32(blob + 20) != F->n_attached || o_get32(blob + 24) != F->n_unattached ||
      F->n_attached < F->n_tracks)
    return O_R_CORRUPT;
  void* dst[O_R_NFIELD] = {o->qpt, o->row, o->slice, o->pad, o->time, o->ncl, o->qtot_a,
                           o->qmax_a, o->flags_a, o->sigma_pad_a, o->sigma_time_a,
                           o->row_diff, o->slice_leg_diff, o->pad_res, o->time_res,
                           o->n_unatt, o->pad_diff_u, o->time_diff_u, o->qtot_u, o->qmax_u,
                           o->flags_u, o->sigma_pad_u, o->sigma_time_u};
  int rc = 0;
  for (int i = 0; i < O_R_NFIELD; i++) {
    const void* a;
    uint32_t w, n;
    o_frame_field(F, i, &a, &w, &n);
    const uint8_t* d = blob + 32 + 32 * i;
    const uint64_t off = o_get64(d), len = o_get64(d + 8);
    if (o_get32(d + 16) != n || o_get32(d + 20) != w ||
        o_get32(d + 24) != (uint32_t)(((uint64_t)n + O_R_CHUNK - 1) / O_R_CHUNK) ||
        off % 16 != 0 || off < O_R_HEAD || off > bytes || len > bytes - off)
      return O_R_CORRUPT;
    if (tmd_oracle_rans_field_decode(blob + off, len, n, w, dst[i]) != 0) rc = O_R_CORRUPT;
  }
  return rc;
}
