/*
 * ecoevo_oracle.c -- plain, slow, single-threaded CPU simulator.
 *
 * TEST INFRASTRUCTURE ONLY (see ecoevo_oracle.h).  Every function below
 * follows one passage of the paper, cited in its comment, in the order the
 * step is stated; no blocking, fusion or reordering.  Build:
 *   gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared ecoevo_oracle.c -lm
 */
#include "ecoevo_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon et al. (SC'11): ten rounds of two    */
/* 32x32->64 multiplies with the Weyl key schedule between rounds.          */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden ratio            */
      k1 += 0xBB67AE85u; /* sqrt(3) - 1             */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void key_of(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1,
                            uint32_t c2, uint32_t c3, int lane) {
  uint32_t ctr[4] = {c0, c1, c2, c3}, key[2], out[4];
  key_of(seed, key);
  or_philox4x32_10(ctr, key, out);
  return out[lane];
}

/* Box-Muller on u = (x + 1/2) 2^-32, computed in double. */
void or_box_muller(uint32_t x1, uint32_t x2, double *z0, double *z1) {
  const double two_m32 = 1.0 / 4294967296.0;
  double u1 = ((double)x1 + 0.5) * two_m32;
  double u2 = ((double)x2 + 0.5) * two_m32;
  double r = sqrt(-2.0 * log(u1));
  double a = 2.0 * M_PI * u2;
  *z0 = r * cos(a);
  *z1 = r * sin(a);
}

/* One Philox draw {j/4, t, tag, id} gives four normals: lanes (0,1) and
 * (2,3) are two Box-Muller pairs; normal j takes pair (j%4)/2, and the cos
 * (even j) or sin (odd j) member. */
double or_normal(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                 uint32_t j) {
  uint32_t ctr[4] = {j >> 2, t, tag, id}, key[2], out[4];
  key_of(seed, key);
  or_philox4x32_10(ctr, key, out);
  int pair = (int)((j & 3u) >> 1);
  double z0, z1;
  or_box_muller(out[2 * pair], out[2 * pair + 1], &z0, &z1);
  return (j & 1u) ? z1 : z0;
}

/* ------------------------------------------------------------------------ */
/* App. B.1: regrowth probability p(x,y) = p_I(x,y) c(x) + c, Eq. (1).      */
/* ------------------------------------------------------------------------ */

/* Climate value of row y (rows are the latitude axis, y = 0 at the top).
 * Linear form: lat_top at the top row to lat_bottom at the bottom row.
 * Paper form: c = (alpha^x + 1) / (alpha + 1) with x = y / (H - 1). */
static double climate(const OrParams *p, int y) {
  double frac = (p->H > 1) ? (double)y / (double)(p->H - 1) : 0.0;
  if (p->lat_mode == 1) return (pow(p->lat_alpha, frac) + 1.0) / (p->lat_alpha + 1.0);
  return p->lat_top + (p->lat_bottom - p->lat_top) * frac;
}

static uint32_t prob_to_threshold(double prob) {
  if (!(prob > 0.0)) return 0u;
  if (prob >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)floor(prob * 4294967296.0);
}

int or_threshold_table(const OrParams *p, uint32_t *thr) {
  for (int y = 0; y < p->H; ++y) {
    double cy = climate(p, y);
    for (int cls = 0; cls < 4; ++cls) {
      double prob = p->p_class[cls] * cy + p->p_spont;
      thr[y * 4 + cls] = prob_to_threshold(prob);
    }
  }
  return 0;
}

static int in_neighbourhood(const OrParams *p, int dy, int dx) {
  if (dy == 0 && dx == 0) return 0;
  int ady = dy < 0 ? -dy : dy, adx = dx < 0 ? -dx : dx;
  if (p->nbr_shape == 1) return ady + adx <= p->nbr_radius;
  return ady <= p->nbr_radius && adx <= p->nbr_radius;
}

static int count_class(const OrParams *p, int n) {
  int cls = 0;
  for (int e = 0; e < 3; ++e)
    if (n >= p->class_edges[e]) cls = e + 1;
  return cls;
}

/* Synchronous pass: every count reads res_old only.  A cell that is a wall
 * or already holds a resource is copied; an empty cell counts the resources
 * in its neighbourhood (cells off the grid count zero), picks its count
 * class and grows iff its Philox word is below the row/class threshold.
 * The word of cell (y, x) at step t is lane x%4 of the draw
 * {x/4, t, TAG_REGROW, y}; every cell-keyed stream uses this layout. */
void or_regrow(const OrParams *p, uint64_t seed, uint32_t t,
               const uint32_t *thr, const uint8_t *res_old,
               const uint8_t *wall, uint8_t *res_new) {
  const int H = p->H, W = p->W, R = p->nbr_radius;
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      int cell = y * W + x;
      if (wall[cell] || res_old[cell]) {
        res_new[cell] = res_old[cell];
        continue;
      }
      int n = 0;
      for (int dy = -R; dy <= R; ++dy) {
        for (int dx = -R; dx <= R; ++dx) {
          if (!in_neighbourhood(p, dy, dx)) continue;
          int yy = y + dy, xx = x + dx;
          if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
          n += res_old[yy * W + xx] ? 1 : 0;
        }
      }
      int cls = count_class(p, n);
      uint32_t u = philox_word(seed, (uint32_t)x >> 2, t, OR_TAG_REGROW,
                               (uint32_t)y, x & 3);
      res_new[cell] = (u < thr[y * 4 + cls]) ? 1 : 0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* App. B.2: the agents.                                                    */
/* ------------------------------------------------------------------------ */

/* Sensorimotor ability: the 7x7 square centred on the agent, three channels
 * (resource, other agent, wall), channel-major then row-major, and the
 * agent's own energy last.  Off-grid cells read as wall. */
void or_observe(const OrParams *p, const uint8_t *res, const uint8_t *wall,
                const int32_t *slot_map, int32_t y, int32_t x, float energy,
                double *obs) {
  const int H = p->H, W = p->W, half = OR_VIEW / 2;
  for (int dy = -half; dy <= half; ++dy) {
    for (int dx = -half; dx <= half; ++dx) {
      int k = (dy + half) * OR_VIEW + (dx + half);
      int yy = y + dy, xx = x + dx;
      double r = 0.0, a = 0.0, wl = 1.0;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
        int cell = yy * W + xx;
        r = res[cell] ? 1.0 : 0.0;
        a = (slot_map[cell] >= 0 && !(dy == 0 && dx == 0)) ? 1.0 : 0.0;
        wl = wall[cell] ? 1.0 : 0.0;
      }
      obs[0 * 49 + k] = r;
      obs[1 * 49 + k] = a;
      obs[2 * 49 + k] = wl;
    }
  }
  obs[147] = (double)energy;
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Cognitive capacity: z = W [obs; h] + b with gates i, f, g, o in blocks of
 * 32 rows; c' = s(f) c + s(i) tanh(g); h' = s(o) tanh(c'); logits =
 * Wo h' + bo; the action is the first index of the largest logit. */
int or_lstm_step(const float *w, const double *obs, double *h, double *c,
                 double *logits) {
  double v[OR_NIN];
  for (int k = 0; k < OR_NOBS; ++k) v[k] = obs[k];
  for (int k = 0; k < OR_HID; ++k) v[OR_NOBS + k] = h[k];
  double z[OR_NGATE];
  for (int r = 0; r < OR_NGATE; ++r) {
    double acc = 0.0;
    for (int k = 0; k < OR_NIN; ++k) acc += (double)w[r * OR_NIN + k] * v[k];
    z[r] = acc + (double)w[OR_OFF_B + r];
  }
  for (int j = 0; j < OR_HID; ++j) {
    double gi = sigmoid(z[0 * OR_HID + j]);
    double gf = sigmoid(z[1 * OR_HID + j]);
    double gg = tanh(z[2 * OR_HID + j]);
    double go = sigmoid(z[3 * OR_HID + j]);
    c[j] = gf * c[j] + gi * gg;
    h[j] = go * tanh(c[j]);
  }
  int best = 0;
  for (int a = 0; a < OR_NACT; ++a) {
    double acc = 0.0;
    for (int j = 0; j < OR_HID; ++j)
      acc += (double)w[OR_OFF_WO + a * OR_HID + j] * h[j];
    logits[a] = acc + (double)w[OR_OFF_BO + a];
    if (logits[a] > logits[best]) best = a;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* The paper's controller, App. B.5.                                        */
/* ------------------------------------------------------------------------ */
int or_param_count(int controller) {
  if (controller == OR_CTRL_LSTM32) return OR_NPARAM;
  if (controller == OR_CTRL_PAPER) return OR_PC_NPARAM;
  return -1;
}

/* Sensorimotor ability with the paper's 15x15 view: resource, other agent
 * (the agent's own cell reads 0) and wall channels; cells off the grid read
 * as wall. */
void or_pc_observe(const OrParams *p, const uint8_t *res, const uint8_t *wall,
                   const int32_t *slot_map, int32_t y, int32_t x, double *obs) {
  const int half = OR_PC_VIEW / 2;
  for (int dy = -half; dy <= half; ++dy) {
    for (int dx = -half; dx <= half; ++dx) {
      double *o = obs + ((dy + half) * OR_PC_VIEW + (dx + half)) * 3;
      int yy = y + dy, xx = x + dx;
      if (yy < 0 || yy >= p->H || xx < 0 || xx >= p->W) {
        o[0] = 0.0; o[1] = 0.0; o[2] = 1.0;
        continue;
      }
      int cell = yy * p->W + xx;
      o[0] = res[cell] ? 1.0 : 0.0;
      o[1] = (slot_map[cell] >= 0 && !(dy == 0 && dx == 0)) ? 1.0 : 0.0;
      o[2] = wall[cell] ? 1.0 : 0.0;
    }
  }
}

/* 3x3 convolution, stride 2, zero padding of one cell on each side ("same"
 * for these sizes): in [n][n][ci], out [m][m][co], weights [co][3][3][ci]. */
static void conv3x3_s2(const double *in, int n, int ci, const float *wt, const float *b,
                       int co, double *out, int m) {
  for (int oy = 0; oy < m; ++oy)
    for (int ox = 0; ox < m; ++ox)
      for (int f = 0; f < co; ++f) {
        double acc = (double)b[f];
        for (int ky = 0; ky < 3; ++ky)
          for (int kx = 0; kx < 3; ++kx) {
            int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
            if (iy < 0 || iy >= n || ix < 0 || ix >= n) continue;
            for (int c = 0; c < ci; ++c)
              acc += (double)wt[((f * 3 + ky) * 3 + kx) * ci + c] * in[(iy * n + ix) * ci + c];
          }
        out[(oy * m + ox) * co + f] = acc;
      }
}

/* 2x2 average pool, stride 1, no padding: [n][n][c] -> [n-1][n-1][c]. */
static void avgpool2_s1(const double *in, int n, int c, double *out) {
  for (int y = 0; y + 1 < n; ++y)
    for (int x = 0; x + 1 < n; ++x)
      for (int k = 0; k < c; ++k)
        out[(y * (n - 1) + x) * c + k] =
            0.25 * (in[(y * n + x) * c + k] + in[(y * n + x + 1) * c + k] +
                    in[((y + 1) * n + x) * c + k] + in[((y + 1) * n + x + 1) * c + k]);
}

void or_pc_forward(const float *w, const double *obs, int prev_action, int ate,
                   double *h, double *c, double *logits) {
  double a1[8 * 8 * 4], p1[7 * 7 * 4], a2[4 * 4 * 8], emb[OR_PC_EMB + OR_PC_HID];
  conv3x3_s2(obs, OR_PC_VIEW, 3, w + OR_PC_W1, w + OR_PC_B1, 4, a1, 8);
  avgpool2_s1(a1, 8, 4, p1);
  conv3x3_s2(p1, 7, 4, w + OR_PC_W2, w + OR_PC_B2, 8, a2, 4);
  avgpool2_s1(a2, 4, 8, emb);                      /* emb[0..71] */
  for (int a = 0; a < OR_NACT; ++a) emb[72 + a] = (a == prev_action) ? 1.0 : 0.0;
  emb[77] = ate ? 1.0 : 0.0;
  /* LSTM, 4 units, gates i, f, g, o */
  double z[4 * OR_PC_HID];
  for (int r = 0; r < 4 * OR_PC_HID; ++r) {
    double acc = (double)w[OR_PC_BL + r];
    for (int k = 0; k < OR_PC_EMB; ++k) acc += (double)w[OR_PC_WI + r * OR_PC_EMB + k] * emb[k];
    for (int j = 0; j < OR_PC_HID; ++j) acc += (double)w[OR_PC_WH + r * OR_PC_HID + j] * h[j];
    z[r] = acc;
  }
  for (int j = 0; j < OR_PC_HID; ++j) {
    double gi = sigmoid(z[0 * OR_PC_HID + j]);
    double gf = sigmoid(z[1 * OR_PC_HID + j]);
    double gg = tanh(z[2 * OR_PC_HID + j]);
    double go = sigmoid(z[3 * OR_PC_HID + j]);
    c[j] = gf * c[j] + gi * gg;
    h[j] = go * tanh(c[j]);
  }
  /* [embedding, h'] -> dense 8, tanh -> dense 5 */
  for (int j = 0; j < OR_PC_HID; ++j) emb[OR_PC_EMB + j] = h[j];
  double d[8];
  for (int i = 0; i < 8; ++i) {
    double acc = (double)w[OR_PC_DB1 + i];
    for (int k = 0; k < OR_PC_EMB + OR_PC_HID; ++k)
      acc += (double)w[OR_PC_D1 + i * (OR_PC_EMB + OR_PC_HID) + k] * emb[k];
    d[i] = tanh(acc);
  }
  for (int a = 0; a < OR_NACT; ++a) {
    double acc = (double)w[OR_PC_DB2 + a];
    for (int i = 0; i < 8; ++i) acc += (double)w[OR_PC_D2 + a * 8 + i] * d[i];
    logits[a] = acc;
  }
}

double or_action_uniform(uint64_t seed, uint32_t t, uint32_t slot) {
  uint32_t word = philox_word(seed, slot, t, OR_TAG_ACT, 0u, 0);
  return (double)(word >> 8) * (1.0 / 16777216.0);
}

int or_pc_sample(const double *logits, double u) {
  double m = logits[0];
  for (int a = 1; a < OR_NACT; ++a) if (logits[a] > m) m = logits[a];
  double e[OR_NACT], sum = 0.0;
  for (int a = 0; a < OR_NACT; ++a) {
    e[a] = exp(OR_PC_INV_TEMP * (logits[a] - m));
    sum += e[a];
  }
  int action = 0;
  double cdf = 0.0;
  for (int k = 0; k < OR_NACT - 1; ++k) {
    cdf += e[k] / sum;
    if (cdf <= u) action = k + 1;
  }
  return action;
}

/* ------------------------------------------------------------------------ */
/* Error magnitudes of the controllers' outputs (test support).             */
/* ------------------------------------------------------------------------ */
/* Not part of the method: these functions give, for every output of one
 * controller step, the first-order magnitude E that bounds how far an
 * evaluation rounding each operation with relative error at most eps can be
 * from the exact (here FP64) result: |computed - exact| <= eps * E, up to
 * second-order terms, when eps covers the longest chain of roundings (a
 * dot product of n terms: about n * 2^-24 in FP32).  It is a running error
 * analysis (Wilkinson; Higham, "Accuracy and Stability of Numerical
 * Algorithms", 2nd ed., sections 3.1-3.3): E of an exactly known input is
 * 0; an input that is a previous step's output carries that step's E; then
 *   dot product  z = b + sum_k w_k v_k:  E_z = |b| + sum_k |w_k| (|v_k| + E_vk)
 *   activation   a = f(z):               E_a = |f'(z)| E_z + |a|
 *   product      p = x y:                E_p = |x| E_y + |y| E_x + |p|
 *   average of four  m = (x1+..+x4)/4:   E_m = (E_1 + E_2 + E_3 + E_4) / 4 + |m|
 *   sum          s = x + y:              E_s = E_x + E_y + |s|
 * (the |.| of an operation's own result, or |b| + sum |w_k v_k| of a dot
 * product, is the rounding of that operation; the rest carries its inputs'
 * magnitudes through the absolute values of the partial derivatives, so E
 * is at least the first-order worst case over every choice of rounding
 * errors).  The parity tests bound each recurrent output and logit of the
 * CUDA path by a tolerance times E. */

/* derivative of the logistic function from its value */
static double dsigmoid_of(double s) { return s * (1.0 - s); }

/* One gate-to-state update of unit j from pre-activations (z, E_z) of its
 * gates i, f, g, o and the previous (c, E_c): writes (c', E_c'), (h', E_h'). */
static void cell_mag(double zi, double ezi, double zf, double ezf, double zg, double ezg,
                     double zo, double ezo, double c, double ec, double *cn, double *ecn,
                     double *hn, double *ehn) {
  const double gi = sigmoid(zi), gf = sigmoid(zf), gg = tanh(zg), go = sigmoid(zo);
  const double ei = dsigmoid_of(gi) * ezi + fabs(gi);
  const double ef = dsigmoid_of(gf) * ezf + fabs(gf);
  const double eg = (1.0 - gg * gg) * ezg + fabs(gg);
  const double eo = dsigmoid_of(go) * ezo + fabs(go);
  const double fc = gf * c, ig = gi * gg;
  *cn = fc + ig;
  *ecn = (fabs(gf) * ec + fabs(c) * ef + fabs(fc)) + (fabs(gi) * eg + fabs(gg) * ei + fabs(ig)) +
         fabs(*cn);
  const double tc = tanh(*cn);
  const double etc = (1.0 - tc * tc) * (*ecn) + fabs(tc);
  *hn = go * tc;
  *ehn = fabs(go) * etc + fabs(tc) * eo + fabs(*hn);
}

void or_lstm_mag(const float *w, const double *obs, const double *h, const double *c,
                 const double *eh, const double *ec, double *eh_out, double *ec_out,
                 double *el_out) {
  double v[OR_NIN], ev[OR_NIN];
  for (int k = 0; k < OR_NOBS; ++k) {
    v[k] = obs[k];
    ev[k] = 0.0;
  }
  for (int k = 0; k < OR_HID; ++k) {
    v[OR_NOBS + k] = h[k];
    ev[OR_NOBS + k] = eh[k];
  }
  double z[OR_NGATE], ez[OR_NGATE];
  for (int r = 0; r < OR_NGATE; ++r) {
    double acc = (double)w[OR_OFF_B + r], e = fabs((double)w[OR_OFF_B + r]);
    for (int k = 0; k < OR_NIN; ++k) {
      const double wk = (double)w[r * OR_NIN + k];
      acc += wk * v[k];
      e += fabs(wk) * (fabs(v[k]) + ev[k]);
    }
    z[r] = acc;
    ez[r] = e;
  }
  double hn[OR_HID], ehn[OR_HID], ecn[OR_HID];
  for (int j = 0; j < OR_HID; ++j) {
    double cn;
    cell_mag(z[j], ez[j], z[OR_HID + j], ez[OR_HID + j], z[2 * OR_HID + j],
             ez[2 * OR_HID + j], z[3 * OR_HID + j], ez[3 * OR_HID + j], c[j], ec[j], &cn,
             &ecn[j], &hn[j], &ehn[j]);
  }
  for (int a = 0; a < OR_NACT; ++a) {
    double e = fabs((double)w[OR_OFF_BO + a]);
    for (int j = 0; j < OR_HID; ++j)
      e += fabs((double)w[OR_OFF_WO + a * OR_HID + j]) * (fabs(hn[j]) + ehn[j]);
    el_out[a] = e;
  }
  for (int j = 0; j < OR_HID; ++j) {
    eh_out[j] = ehn[j];
    ec_out[j] = ecn[j];
  }
}

/* conv3x3_s2 with magnitudes: E_in [n][n][ci] -> E_out [m][m][co] */
static void conv3x3_s2_mag(const double *in, const double *ein, int n, int ci, const float *wt,
                           const float *b, int co, double *out, double *eout, int m) {
  for (int oy = 0; oy < m; ++oy)
    for (int ox = 0; ox < m; ++ox)
      for (int f = 0; f < co; ++f) {
        double acc = (double)b[f], e = fabs((double)b[f]);
        for (int ky = 0; ky < 3; ++ky)
          for (int kx = 0; kx < 3; ++kx) {
            int iy = 2 * oy + ky - 1, ix = 2 * ox + kx - 1;
            if (iy < 0 || iy >= n || ix < 0 || ix >= n) continue;
            for (int cc = 0; cc < ci; ++cc) {
              const double wk = (double)wt[((f * 3 + ky) * 3 + kx) * ci + cc];
              const int i = (iy * n + ix) * ci + cc;
              acc += wk * in[i];
              e += fabs(wk) * (fabs(in[i]) + ein[i]);
            }
          }
        out[(oy * m + ox) * co + f] = acc;
        eout[(oy * m + ox) * co + f] = e;
      }
}

/* avgpool2_s1 of the magnitudes; out: the pooled values (avgpool2_s1) */
static void avgpool2_s1_mag(const double *ein, int n, int c, const double *out, double *eout) {
  for (int y = 0; y + 1 < n; ++y)
    for (int x = 0; x + 1 < n; ++x)
      for (int k = 0; k < c; ++k) {
        const int o = (y * (n - 1) + x) * c + k;
        eout[o] = 0.25 * (ein[(y * n + x) * c + k] + ein[(y * n + x + 1) * c + k] +
                          ein[((y + 1) * n + x) * c + k] + ein[((y + 1) * n + x + 1) * c + k]) +
                  fabs(out[o]);
      }
}

void or_pc_mag(const float *w, const double *obs, int prev_action, int ate, const double *h,
               const double *c, const double *eh, const double *ec, double *eh_out,
               double *ec_out, double *el_out) {
  static const double zero_obs[OR_PC_NOBS];   /* the view is exact */
  double a1[8 * 8 * 4], ea1[8 * 8 * 4], p1[7 * 7 * 4], ep1[7 * 7 * 4];
  double a2[4 * 4 * 8], ea2[4 * 4 * 8];
  double emb[OR_PC_EMB + OR_PC_HID], eemb[OR_PC_EMB + OR_PC_HID];
  conv3x3_s2_mag(obs, zero_obs, OR_PC_VIEW, 3, w + OR_PC_W1, w + OR_PC_B1, 4, a1, ea1, 8);
  avgpool2_s1(a1, 8, 4, p1);
  avgpool2_s1_mag(ea1, 8, 4, p1, ep1);
  conv3x3_s2_mag(p1, ep1, 7, 4, w + OR_PC_W2, w + OR_PC_B2, 8, a2, ea2, 4);
  avgpool2_s1(a2, 4, 8, emb);
  avgpool2_s1_mag(ea2, 4, 8, emb, eemb);
  for (int a = 0; a < OR_NACT; ++a) {
    emb[72 + a] = (a == prev_action) ? 1.0 : 0.0;
    eemb[72 + a] = 0.0;
  }
  emb[77] = ate ? 1.0 : 0.0;
  eemb[77] = 0.0;
  double z[4 * OR_PC_HID], ez[4 * OR_PC_HID];
  for (int r = 0; r < 4 * OR_PC_HID; ++r) {
    double acc = (double)w[OR_PC_BL + r], e = fabs((double)w[OR_PC_BL + r]);
    for (int k = 0; k < OR_PC_EMB; ++k) {
      const double wk = (double)w[OR_PC_WI + r * OR_PC_EMB + k];
      acc += wk * emb[k];
      e += fabs(wk) * (fabs(emb[k]) + eemb[k]);
    }
    for (int j = 0; j < OR_PC_HID; ++j) {
      const double wk = (double)w[OR_PC_WH + r * OR_PC_HID + j];
      acc += wk * h[j];
      e += fabs(wk) * (fabs(h[j]) + eh[j]);
    }
    z[r] = acc;
    ez[r] = e;
  }
  double ehn[OR_PC_HID], ecn[OR_PC_HID];
  for (int j = 0; j < OR_PC_HID; ++j) {
    double cn, hn;
    cell_mag(z[j], ez[j], z[OR_PC_HID + j], ez[OR_PC_HID + j], z[2 * OR_PC_HID + j],
             ez[2 * OR_PC_HID + j], z[3 * OR_PC_HID + j], ez[3 * OR_PC_HID + j], c[j], ec[j],
             &cn, &ecn[j], &hn, &ehn[j]);
    emb[OR_PC_EMB + j] = hn;
    eemb[OR_PC_EMB + j] = ehn[j];
  }
  double d[8], ed[8];
  for (int i = 0; i < 8; ++i) {
    double acc = (double)w[OR_PC_DB1 + i], e = fabs((double)w[OR_PC_DB1 + i]);
    for (int k = 0; k < OR_PC_EMB + OR_PC_HID; ++k) {
      const double wk = (double)w[OR_PC_D1 + i * (OR_PC_EMB + OR_PC_HID) + k];
      acc += wk * emb[k];
      e += fabs(wk) * (fabs(emb[k]) + eemb[k]);
    }
    d[i] = tanh(acc);
    ed[i] = (1.0 - d[i] * d[i]) * e + fabs(d[i]);
  }
  for (int a = 0; a < OR_NACT; ++a) {
    double e = fabs((double)w[OR_PC_DB2 + a]);
    for (int i = 0; i < 8; ++i) e += fabs((double)w[OR_PC_D2 + a * 8 + i]) * (fabs(d[i]) + ed[i]);
    el_out[a] = e;
  }
  for (int j = 0; j < OR_PC_HID; ++j) {
    eh_out[j] = ehn[j];
    ec_out[j] = ecn[j];
  }
}

/* ------------------------------------------------------------------------ */
/* The world.                                                               */
/* ------------------------------------------------------------------------ */
struct OrWorld {
  OrParams p;
  uint64_t seed;
  uint8_t *res, *wall, *res_tmp;
  int32_t *slot_map;
  uint8_t *alive, *ate, *killed, *wants;
  int32_t *y, *x, *repr_ctr, *low_ctr, *age, *action, *target, *cand;
  int32_t *claim, *birth_parent, *birth_child, *free_list, *move_action, *prev_act;
  /* lab-environment greediness (App. C): per slot, bit 0 = a resource was in
   * view during the current window, bit 1 = ate during it; windows with a
   * resource in view (T_r) and with a consumption (C_r) */
  uint8_t *lab_flags;
  int32_t *lab_t, *lab_c;
  float *energy, *weights;
  double *h, *c, *logits;
  /* test support: error magnitudes of h, c and the logits (or_lstm_mag),
   * computed while track_mag is set (the default) */
  double *mag_h, *mag_c, *mag_l;
  int track_mag;
  uint32_t *thr;
  int64_t counters[OR_NCOUNTERS];
  /* analysis metrics, App. C: an identity for every agent (-1: empty slot),
   * the identities and cells at the start of the current window, and the
   * deaths and summed ages at death since then */
  int64_t *agent_id, *snap_id;
  int32_t *snap_cell;
  int64_t next_id, snap_t, an_deaths, an_age_sum;
  /* visiting order of the per-slot loops whose outcome the method leaves
   * independent of it (NULL: ascending); a test hook, or_world_set_order */
  int32_t *order;
};

/* Slot visited i-th by those loops. */
static int slot_at(const OrWorld *w, int i) { return w->order ? w->order[i] : i; }

static const int DY[5] = {0, -1, 1, 0, 0}; /* stay, N, S, E, W */
static const int DX[5] = {0, 0, 0, 1, -1};

void *or_world_field(OrWorld *w, int f) {
  switch (f) {
    case OR_F_RES: return w->res;
    case OR_F_WALL: return w->wall;
    case OR_F_SLOT_MAP: return w->slot_map;
    case OR_F_ALIVE: return w->alive;
    case OR_F_Y: return w->y;
    case OR_F_X: return w->x;
    case OR_F_ENERGY: return w->energy;
    case OR_F_REPR_CTR: return w->repr_ctr;
    case OR_F_LOW_CTR: return w->low_ctr;
    case OR_F_AGE: return w->age;
    case OR_F_H: return w->h;
    case OR_F_C: return w->c;
    case OR_F_ACTION: return w->action;
    case OR_F_LOGITS: return w->logits;
    case OR_F_ATE: return w->ate;
    case OR_F_WEIGHTS: return w->weights;
    case OR_F_COUNTERS: return w->counters;
    case OR_F_THR: return w->thr;
    case OR_F_BIRTH_PARENT: return w->birth_parent;
    case OR_F_BIRTH_CHILD: return w->birth_child;
    case OR_F_MOVE_ACTION: return w->move_action;
    case OR_F_PREV_ACTION: return w->prev_act;
    case OR_F_LAB_FLAGS: return w->lab_flags;
    case OR_F_LAB_T: return w->lab_t;
    case OR_F_LAB_C: return w->lab_c;
    case OR_F_MAG_H: return w->mag_h;
    case OR_F_MAG_C: return w->mag_c;
    case OR_F_MAG_LOGITS: return w->mag_l;
    default: return NULL;
  }
}

void or_world_destroy(OrWorld *w) {
  if (!w) return;
  free(w->res); free(w->wall); free(w->res_tmp); free(w->slot_map);
  free(w->alive); free(w->ate); free(w->killed); free(w->wants);
  free(w->y); free(w->x); free(w->repr_ctr); free(w->low_ctr); free(w->age);
  free(w->action); free(w->target); free(w->cand); free(w->claim);
  free(w->birth_parent); free(w->birth_child); free(w->free_list);
  free(w->move_action); free(w->prev_act);
  free(w->lab_flags); free(w->lab_t); free(w->lab_c);
  free(w->energy); free(w->weights); free(w->h); free(w->c); free(w->logits);
  free(w->mag_h); free(w->mag_c); free(w->mag_l);
  free(w->thr);
  free(w->agent_id); free(w->snap_id); free(w->snap_cell);
  free(w->order);
  free(w);
}

void or_world_track_magnitudes(OrWorld *w, int on) { w->track_mag = on ? 1 : 0; }

int or_world_set_order(OrWorld *w, const int32_t *perm) {
  const int C = w->p.capacity;
  if (!perm) {
    free(w->order);
    w->order = NULL;
    return 0;
  }
  uint8_t *seen = calloc(C > 0 ? C : 1, 1);
  int32_t *copy = malloc((C > 0 ? C : 1) * sizeof(int32_t));
  if (!seen || !copy) {
    free(seen);
    free(copy);
    return -2;
  }
  for (int i = 0; i < C; ++i) {
    if (perm[i] < 0 || perm[i] >= C || seen[perm[i]]) {
      free(seen);
      free(copy);
      return -1;
    }
    seen[perm[i]] = 1;
    copy[i] = perm[i];
  }
  free(seen);
  free(w->order);
  w->order = copy;
  return 0;
}

static int valid_params(const OrParams *p) {
  if (p->H < 1 || p->W < 1 || p->capacity < 0 || p->n_agents0 < 0) return 0;
  if (p->n_agents0 > p->capacity) return 0;
  if (p->nbr_radius < 1 || p->nbr_radius > 3) return 0;
  if (p->nbr_shape != 0 && p->nbr_shape != 1) return 0;
  if (p->lat_mode != 0 && p->lat_mode != 1) return 0;
  if (or_param_count(p->controller) < 0) return 0;
  return 1;
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

/* out[j] = base[j] + scale * N_j for j < 23333 (base NULL reads as zero),
 * with N_j normal j of the stream (seed, tag, t, id); one Philox draw serves
 * the four normals 4q..4q+3, as or_normal defines them. */
void or_fill_normals(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                     float scale, const float *base, float *out) {
  or_fill_normals_n(seed, tag, t, id, scale, base, out, OR_NPARAM);
}

void or_fill_normals_n(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                       float scale, const float *base, float *out, int n) {
  uint32_t key[2];
  key_of(seed, key);
  for (uint32_t q = 0; 4 * q < (uint32_t)n; ++q) {
    uint32_t ctr[4] = {q, t, tag, id}, r[4];
    or_philox4x32_10(ctr, key, r);
    double z[4];
    or_box_muller(r[0], r[1], &z[0], &z[1]);
    or_box_muller(r[2], r[3], &z[2], &z[3]);
    for (uint32_t i = 0; i < 4 && 4 * q + i < (uint32_t)n; ++i) {
      uint32_t j = 4 * q + i;
      double b = base ? (double)base[j] : 0.0;
      out[j] = (float)(b + (double)scale * z[i]);
    }
  }
}

int or_initial_layout(const OrParams *p, uint64_t seed, uint8_t *res, uint8_t *wall,
                      int32_t *cells) {
  if (!valid_params(p)) return -1;
  const int H = p->H, W = p->W;
  const size_t HW = (size_t)H * (size_t)W;

  /* Border walls (App. B.1 environment: walls are cells agents cannot
   * cross). */
  for (int yy = 0; yy < H; ++yy)
    for (int xx = 0; xx < W; ++xx)
      wall[yy * W + xx] =
          (p->border_walls && (yy == 0 || yy == H - 1 || xx == 0 || xx == W - 1)) ? 1 : 0;

  /* Initial resources: Bernoulli(res_init_p) on every non-wall cell. */
  uint32_t thr_init = prob_to_threshold(p->res_init_p);
  for (size_t cell = 0; cell < HW; ++cell) {
    res[cell] = 0;
    if (wall[cell]) continue;
    uint32_t u = philox_word(seed, (uint32_t)(cell % W) >> 2, 0u, OR_TAG_RES_INIT,
                             (uint32_t)(cell / W), (int)(cell % W) & 3);
    res[cell] = (u < thr_init) ? 1 : 0;
  }

  /* Random placement: the non-wall cells sorted by (Philox word, cell); the
   * first n_agents0 cells receive slots 0.. in that order. */
  size_t nfree = 0;
  for (size_t cell = 0; cell < HW; ++cell) nfree += wall[cell] ? 0 : 1;
  if ((size_t)p->n_agents0 > nfree) return -1;
  if (p->n_agents0 == 0) return 0;
  uint64_t *keys = malloc(nfree * sizeof(uint64_t));
  if (!keys) return -2;
  size_t k = 0;
  for (size_t cell = 0; cell < HW; ++cell) {
    if (wall[cell]) continue;
    uint32_t u = philox_word(seed, (uint32_t)(cell % W) >> 2, 0u, OR_TAG_PLACE,
                             (uint32_t)(cell / W), (int)(cell % W) & 3);
    keys[k++] = ((uint64_t)u << 32) | (uint64_t)cell;
  }
  qsort(keys, nfree, sizeof(uint64_t), cmp_u64);
  for (int s = 0; s < p->n_agents0; ++s) cells[s] = (int32_t)(keys[s] & 0xFFFFFFFFu);
  free(keys);
  return 0;
}

/* A fresh identity for every living agent, and a new analysis window that
 * starts at the current state. */
static void take_snapshot(OrWorld *w) {
  for (int s = 0; s < w->p.capacity; ++s) {
    w->snap_id[s] = w->agent_id[s];
    w->snap_cell[s] = w->alive[s] ? w->y[s] * w->p.W + w->x[s] : -1;
  }
  w->snap_t = w->counters[OR_C_T];
  w->an_deaths = 0;
  w->an_age_sum = 0;
}

static void new_identities(OrWorld *w) {
  w->next_id = 0;
  for (int s = 0; s < w->p.capacity; ++s)
    w->agent_id[s] = w->alive[s] ? w->next_id++ : -1;
  take_snapshot(w);
}

int or_world_create(const OrParams *p, uint64_t seed, OrWorld **out) {
  *out = NULL;
  if (!valid_params(p)) return -1;
  OrWorld *w = (OrWorld *)calloc(1, sizeof(OrWorld));
  if (!w) return -2;
  w->p = *p;
  w->seed = seed;
  w->track_mag = 1;
  const size_t HW = (size_t)p->H * (size_t)p->W, C = (size_t)p->capacity;
  const size_t C1 = C ? C : 1;
  w->res = calloc(HW, 1); w->wall = calloc(HW, 1); w->res_tmp = calloc(HW, 1);
  w->slot_map = malloc(HW * sizeof(int32_t));
  w->claim = malloc(HW * sizeof(int32_t));
  w->alive = calloc(C1, 1); w->ate = calloc(C1, 1);
  w->killed = calloc(C1, 1); w->wants = calloc(C1, 1);
  w->y = calloc(C1, 4); w->x = calloc(C1, 4); w->repr_ctr = calloc(C1, 4);
  w->low_ctr = calloc(C1, 4); w->age = calloc(C1, 4); w->action = calloc(C1, 4);
  w->target = calloc(C1, 4); w->cand = calloc(C1, 4);
  w->birth_parent = calloc(C1, 4); w->birth_child = calloc(C1, 4);
  w->free_list = calloc(C1, 4);
  w->move_action = calloc(C1, 4);
  w->prev_act = calloc(C1, 4);
  w->lab_flags = calloc(C1, 1);
  w->lab_t = calloc(C1, 4);
  w->lab_c = calloc(C1, 4);
  w->energy = calloc(C1, sizeof(float));
  w->weights = calloc(C1 * OR_NPARAM, sizeof(float));
  w->h = calloc(C1 * OR_HID, sizeof(double));
  w->c = calloc(C1 * OR_HID, sizeof(double));
  w->logits = calloc(C1 * OR_NACT, sizeof(double));
  w->mag_h = calloc(C1 * OR_HID, sizeof(double));
  w->mag_c = calloc(C1 * OR_HID, sizeof(double));
  w->mag_l = calloc(C1 * OR_NACT, sizeof(double));
  w->thr = calloc((size_t)p->H * 4, sizeof(uint32_t));
  w->agent_id = malloc(C1 * sizeof(int64_t));
  w->snap_id = malloc(C1 * sizeof(int64_t));
  w->snap_cell = malloc(C1 * sizeof(int32_t));
  if (!w->agent_id || !w->snap_id || !w->snap_cell || !w->res || !w->wall || !w->res_tmp || !w->slot_map || !w->claim ||
      !w->alive || !w->ate || !w->killed || !w->wants || !w->y || !w->x ||
      !w->repr_ctr || !w->low_ctr || !w->age || !w->action || !w->target ||
      !w->cand || !w->birth_parent || !w->birth_child || !w->free_list || !w->move_action ||
      !w->prev_act || !w->lab_flags || !w->lab_t || !w->lab_c ||
      !w->energy || !w->weights || !w->h || !w->c || !w->logits || !w->thr ||
      !w->mag_h || !w->mag_c || !w->mag_l) {
    or_world_destroy(w);
    return -2;
  }
  or_threshold_table(p, w->thr);
  const int W = p->W;
  for (size_t cell = 0; cell < HW; ++cell) {
    w->slot_map[cell] = -1;
    w->claim[cell] = -1;
  }
  int32_t *cells = malloc(((size_t)p->n_agents0 + 1) * sizeof(int32_t));
  if (!cells) { or_world_destroy(w); return -2; }
  int rc = or_initial_layout(p, seed, w->res, w->wall, cells);
  if (rc != 0) {
    free(cells);
    or_world_destroy(w);
    return rc;
  }
  for (int s = 0; s < p->n_agents0; ++s) {
    const int32_t cell = cells[s];
    w->alive[s] = 1;
    w->y[s] = cell / W;
    w->x[s] = cell % W;
    w->slot_map[cell] = s;
    w->energy[s] = p->e0;
    /* weights drawn once at the start of the simulation, App. B.2 */
    or_fill_normals_n(seed, OR_TAG_INIT_W, 0u, (uint32_t)s, p->w_init_std, NULL,
                      w->weights + (size_t)s * OR_NPARAM, or_param_count(p->controller));
  }
  free(cells);
  w->counters[OR_C_POP] = p->n_agents0;
  new_identities(w);
  *out = w;
  return 0;
}

int or_world_sync(OrWorld *w) {
  const OrParams *p = &w->p;
  const int H = p->H, W = p->W;
  or_threshold_table(p, w->thr);
  for (int i = 0; i < H * W; ++i) w->slot_map[i] = -1;
  int64_t pop = 0;
  for (int s = 0; s < p->capacity; ++s) {
    if (!w->alive[s]) continue;
    int yy = w->y[s], xx = w->x[s];
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) return -1;
    int cell = yy * W + xx;
    if (w->wall[cell] || w->slot_map[cell] >= 0 || w->age[s] < 0) return -1;
    w->slot_map[cell] = s;
    ++pop;
  }
  w->counters[OR_C_POP] = pop;
  new_identities(w);
  for (int s = 0; s < p->capacity; ++s) {
    w->lab_flags[s] = 0;
    w->lab_t[s] = 0;
    w->lab_c[s] = 0;
  }
  /* written state is exact */
  memset(w->mag_h, 0, (size_t)(p->capacity ? p->capacity : 1) * OR_HID * sizeof(double));
  memset(w->mag_c, 0, (size_t)(p->capacity ? p->capacity : 1) * OR_HID * sizeof(double));
  memset(w->mag_l, 0, (size_t)(p->capacity ? p->capacity : 1) * OR_NACT * sizeof(double));
  return 0;
}

static int in_grid(const OrParams *p, int yy, int xx) {
  return yy >= 0 && yy < p->H && xx >= 0 && xx < p->W;
}

/* One simulation step.  Order of the parts: regrowth (App. B.1), observation
 * and controller (App. B.2), moves with one claim round, eating, physiology
 * (App. B.2 physiology), death and reproduction (App. B.3). */
int or_world_step(OrWorld *w, const int32_t *forced) {
  const OrParams *p = &w->p;
  const int H = p->H, W = p->W, C = p->capacity;
  const uint32_t t = (uint32_t)w->counters[OR_C_T];
  /* agent-steps: every agent alive at the start of the step takes one */
  w->counters[OR_C_AGENT_STEPS] += w->counters[OR_C_POP];

  /* 1. regrowth from the grid as it stood at the start of the step */
  or_regrow(p, w->seed, t, w->thr, w->res, w->wall, w->res_tmp);
  memcpy(w->res, w->res_tmp, (size_t)H * W);

  /* 2-3. observation (new resources, start-of-step occupancy) and one
   * controller step per living agent */
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    const int ate_last = w->ate[s];   /* the paper controller's input */
    w->ate[s] = 0;
    w->killed[s] = 0;
    w->wants[s] = 0;
    w->target[s] = -1;
    w->cand[s] = -1;
    if (!w->alive[s]) continue;
    if (p->controller == OR_CTRL_PAPER) {
      /* App. B.5: CNN embedding, LSTM(4), dense layers, then an action
       * sampled from the softmax at temperature 1/50 */
      double obs[OR_PC_NOBS];
      or_pc_observe(p, w->res, w->wall, w->slot_map, w->y[s], w->x[s], obs);
      for (int k = 0; k < OR_PC_VIEW * OR_PC_VIEW; ++k)
        if (obs[3 * k] != 0.0) w->lab_flags[s] |= 1;   /* a resource in view */
      if (w->track_mag)
        or_pc_mag(w->weights + (size_t)s * OR_NPARAM, obs, w->prev_act[s], ate_last,
                w->h + (size_t)s * OR_HID, w->c + (size_t)s * OR_HID,
                w->mag_h + (size_t)s * OR_HID, w->mag_c + (size_t)s * OR_HID,
                w->mag_h + (size_t)s * OR_HID, w->mag_c + (size_t)s * OR_HID,
                w->mag_l + (size_t)s * OR_NACT);
      or_pc_forward(w->weights + (size_t)s * OR_NPARAM, obs, w->prev_act[s], ate_last,
                    w->h + (size_t)s * OR_HID, w->c + (size_t)s * OR_HID,
                    w->logits + (size_t)s * OR_NACT);
      w->action[s] = or_pc_sample(w->logits + (size_t)s * OR_NACT,
                                  or_action_uniform(w->seed, t, (uint32_t)s));
      continue;
    }
    double obs[OR_NOBS];
    or_observe(p, w->res, w->wall, w->slot_map, w->y[s], w->x[s], w->energy[s],
               obs);
    for (int k = 0; k < OR_VIEW * OR_VIEW; ++k)
      if (obs[k] != 0.0) w->lab_flags[s] |= 1;     /* a resource in view */
    if (w->track_mag)
      or_lstm_mag(w->weights + (size_t)s * OR_NPARAM, obs, w->h + (size_t)s * OR_HID,
                w->c + (size_t)s * OR_HID, w->mag_h + (size_t)s * OR_HID,
                w->mag_c + (size_t)s * OR_HID, w->mag_h + (size_t)s * OR_HID,
                w->mag_c + (size_t)s * OR_HID, w->mag_l + (size_t)s * OR_NACT);
    w->action[s] = or_lstm_step(w->weights + (size_t)s * OR_NPARAM, obs,
                                w->h + (size_t)s * OR_HID,
                                w->c + (size_t)s * OR_HID,
                                w->logits + (size_t)s * OR_NACT);
  }

  /* 4. moves: a target is valid if on the grid, not a wall and empty at the
   * start of the phase; among valid claimants of a cell the lowest slot
   * moves, every other agent stays. */
  for (int i = 0; i < H * W; ++i) w->claim[i] = -1;
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    w->move_action[s] = 0;
    if (!w->alive[s]) continue;
    int a = forced ? forced[s] : w->action[s];
    w->move_action[s] = a;
    w->prev_act[s] = (a >= 0 && a < OR_NACT) ? a : 0;
    if (a <= 0 || a >= OR_NACT) continue;
    int ty = w->y[s] + DY[a], tx = w->x[s] + DX[a];
    if (!in_grid(p, ty, tx) || w->wall[ty * W + tx]) {
      if (p->wall_kills) w->killed[s] = 1;
      continue;
    }
    int cell = ty * W + tx;
    if (w->slot_map[cell] != -1) continue;
    w->target[s] = cell;
    if (w->claim[cell] == -1 || s < w->claim[cell]) w->claim[cell] = s;
  }
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    int cell = w->target[s];
    if (cell < 0 || w->claim[cell] != s) continue;
    w->slot_map[w->y[s] * W + w->x[s]] = -1;
    w->slot_map[cell] = s;
    w->y[s] = cell / W;
    w->x[s] = cell % W;
  }

  /* 5. eating: an agent on a resource cell consumes it */
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    if (!w->alive[s] || w->killed[s]) continue;
    int cell = w->y[s] * W + w->x[s];
    if (w->res[cell]) {
      w->res[cell] = 0;
      w->ate[s] = 1;
      w->lab_flags[s] |= 2;
    }
  }

  /* 6. physiology: gain when eating, linear decay, clip at e_max; death
   * after t_death consecutive steps at or below e_death (at least one) or
   * past the maximum age; reproduction counter above e_repr. */
  int64_t deaths = 0;
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    if (!w->alive[s]) continue;
    int dead = 0;
    if (w->killed[s]) {
      dead = 1;
    } else {
      float e = w->energy[s];
      if (w->ate[s]) e = e + p->e_gain;
      e = e - p->e_decay;
      if (e > p->e_max) e = p->e_max;
      w->energy[s] = e;
      w->age[s] += 1;
      w->low_ctr[s] = (e <= p->e_death) ? w->low_ctr[s] + 1 : 0;
      int need = p->t_death > 1 ? p->t_death : 1;
      if (w->low_ctr[s] >= need || w->age[s] > p->max_age) dead = 1;
    }
    if (dead) {
      w->alive[s] = 0;
      w->slot_map[w->y[s] * W + w->x[s]] = -1;
      ++deaths;
      w->an_deaths += 1;
      w->an_age_sum += w->age[s];   /* age at death, App. C */
      w->agent_id[s] = -1;
      continue;
    }
    w->repr_ctr[s] = (w->energy[s] > p->e_repr) ? w->repr_ctr[s] + 1 : 0;
    w->wants[s] = (w->repr_ctr[s] >= p->t_repr) ? 1 : 0;
  }

  /* 7. reproduction: each parent takes its first free neighbour in the order
   * N, S, E, W (occupancy after moves and deaths); the lowest parent slot
   * wins a contested cell; the k-th successful parent (ascending) gets the
   * k-th free slot (ascending); births past the free slots are dropped. */
  for (int i = 0; i < H * W; ++i) w->claim[i] = -1;
  for (int i = 0; i < C; ++i) {
    const int s = slot_at(w, i);
    if (!w->alive[s] || !w->wants[s]) continue;
    for (int a = 1; a < OR_NACT; ++a) {
      int ny = w->y[s] + DY[a], nx = w->x[s] + DX[a];
      if (!in_grid(p, ny, nx)) continue;
      int cell = ny * W + nx;
      if (w->wall[cell] || w->slot_map[cell] != -1) continue;
      w->cand[s] = cell;
      break;
    }
    int cell = w->cand[s];
    if (cell >= 0 && (w->claim[cell] == -1 || s < w->claim[cell]))
      w->claim[cell] = s;
  }
  int nfree = 0;
  for (int s = 0; s < C; ++s)
    if (!w->alive[s]) w->free_list[nfree++] = s;
  int k = 0;
  int64_t dropped = 0;
  for (int parent = 0; parent < C; ++parent) {
    int cell = w->cand[parent];
    if (cell < 0 || w->claim[cell] != parent) continue;
    if (k >= nfree) {
      ++dropped;
      continue;
    }
    int child = w->free_list[k];
    w->birth_parent[k] = parent;
    w->birth_child[k] = child;
    ++k;
    w->alive[child] = 1;
    w->agent_id[child] = w->next_id++;
    w->y[child] = cell / W;
    w->x[child] = cell % W;
    w->slot_map[cell] = child;
    w->energy[child] = p->e0;
    w->repr_ctr[child] = 0;
    w->low_ctr[child] = 0;
    w->age[child] = 0;
    w->action[child] = 0;
    w->prev_act[child] = 0;
    w->lab_flags[child] = 0;
    w->lab_t[child] = 0;
    w->lab_c[child] = 0;
    w->ate[child] = 0;
    for (int j = 0; j < OR_HID; ++j) {
      w->h[(size_t)child * OR_HID + j] = 0.0;
      w->c[(size_t)child * OR_HID + j] = 0.0;
    }
    for (int a = 0; a < OR_NACT; ++a) w->logits[(size_t)child * OR_NACT + a] = 0.0;
    for (int j = 0; j < OR_HID; ++j) {
      w->mag_h[(size_t)child * OR_HID + j] = 0.0;
      w->mag_c[(size_t)child * OR_HID + j] = 0.0;
    }
    for (int a = 0; a < OR_NACT; ++a) w->mag_l[(size_t)child * OR_NACT + a] = 0.0;
    /* asexual reproduction: parent weights plus N(0, sigma) noise, App. B.3 */
    or_fill_normals_n(w->seed, OR_TAG_MUT, t, (uint32_t)parent, p->mut_std,
                      w->weights + (size_t)parent * OR_NPARAM,
                      w->weights + (size_t)child * OR_NPARAM, or_param_count(p->controller));
    w->repr_ctr[parent] = 0;
  }

  w->counters[OR_C_T] += 1;
  w->counters[OR_C_POP] += (int64_t)k - deaths;
  w->counters[OR_C_BIRTHS] += k;
  w->counters[OR_C_DEATHS] += deaths;
  w->counters[OR_C_DROPPED] += dropped;
  w->counters[OR_C_BIRTHS_LAST] = k;
  w->counters[OR_C_DEATHS_LAST] = deaths;
  w->counters[OR_C_DROPPED_LAST] = dropped;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Metrics of the analyses, App. C.                                         */
/* ------------------------------------------------------------------------ */
int or_world_analysis(OrWorld *w, int64_t *out) {
  const OrParams *p = &w->p;
  const int W = p->W;
  for (int i = 0; i < OR_NANALYSIS; ++i) out[i] = 0;
  const int64_t t = w->counters[OR_C_T];
  const int64_t len = t - w->snap_t;
  out[OR_A_T] = t;
  out[OR_A_WINDOW] = len;
  /* population size: agents alive */
  for (int s = 0; s < p->capacity; ++s) out[OR_A_POP] += w->alive[s];
  /* amount of resources: the resource channel summed over the grid */
  for (int i = 0; i < p->H * W; ++i) out[OR_A_RES] += w->res[i];
  /* deaths of the window and their ages, for the life expectancy */
  out[OR_A_DEATHS] = w->an_deaths;
  out[OR_A_AGE_SUM] = w->an_age_sum;
  /* movement: each agent alive over the whole window (the same identity at
   * its start and now), Manhattan distance between its cells then and now,
   * counted in 17 equal bins of the len+1 possible distances */
  for (int s = 0; s < p->capacity; ++s) {
    if (!w->alive[s] || w->agent_id[s] < 0 || w->agent_id[s] != w->snap_id[s]) continue;
    const int y0 = w->snap_cell[s] / W, x0 = w->snap_cell[s] % W;
    const int64_t d = llabs((long long)w->y[s] - y0) + llabs((long long)w->x[s] - x0);
    int64_t bin = d * OR_MOVE_BINS / (len + 1);
    if (bin > OR_MOVE_BINS - 1) bin = OR_MOVE_BINS - 1;
    out[OR_A_MOVERS] += 1;
    out[OR_A_BINS + bin] += 1;
  }
  take_snapshot(w);
  return 0;
}

/* Greediness of the lab environments (App. C): a window ends now; every
 * living agent counts it in T_r if a resource was in its view at some step
 * of the window and in C_r if it ate during it. */
void or_world_lab_window(OrWorld *w) {
  for (int s = 0; s < w->p.capacity; ++s) {
    if (w->alive[s]) {
      w->lab_t[s] += w->lab_flags[s] & 1;
      w->lab_c[s] += (w->lab_flags[s] >> 1) & 1;
    }
    w->lab_flags[s] = 0;
  }
}
