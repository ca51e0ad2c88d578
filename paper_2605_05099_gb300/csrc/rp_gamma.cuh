// Gamma and beta samplers as word-fed state machines (included by
// rp_kernels.cu).
//
// Gamma(alpha, 1) by Marsaglia & Tsang (Randompack Sec. 3.1, gamma): with
// d = s - 1/3 and c = 1/sqrt(9 d), an attempt draws x ~ N(0,1) (the ziggurat
// of Sec. 3.1), sets v = 1 + c x and starts over if v <= 0, else sets v = v^3,
// draws U and accepts d v when U < 1 - 0.0331 x^4 or
// log U < x^2/2 + d (1 - v + log v).  For alpha < 1 the attempt runs with
// s = alpha + 1 and the accepted value is boosted by U'^(1/alpha) with one
// more word.  Beta(a, b) = X / (X + Y) with X ~ Gamma(a) drawn before
// Y ~ Gamma(b) (Table "continuous", beta).
//
// Every accept decision is first made in FP32 with an error margin and
// otherwise by the exact FP64 arithmetic of the serial definition (with
// correctly rounded logs).  The output value of a variate is a function of a
// small record of words (the accepted normal word(s) and the boost word), so
// it is evaluated later, when whole rows of outputs are written.
//
// This file is a fragment of rp_kernels.cu: it is included inside that file's
// namespace, after wedge_accept() and tail_pair_accept().

constexpr double kSqueeze = 0.0331;

// Accepted normal: kind 1 -> value from the word xa; kind 2 -> tail value
// from the candidate word xa (sign) and the accepted pair's first word xb.
__device__ __forceinline__ double normal_x_exact(int xk, u64 xa, u64 xb, const ZigDev& z) {
  if (xk == 1) {
    int i = (int)(xa & 0xff);
    return neg_if(mul_rn_dmul((xa >> 9) & ((1ull << 52) - 1), z.w[i]), (xa >> 8) & 1);
  }
  double a = __ddiv_rn(-cr_log_nl(__dsub_rn(1.0, u53_bits(xb))), z.R);
  return neg_if(__dadd_rn(z.R, a), (xa >> 8) & 1);
}

// FP32 estimate of the same x: relative error below 2^-20.
__device__ __forceinline__ float normal_x_f(int xk, u64 xa, u64 xb, const ZigDev& z) {
  float x;
  if (xk == 1) {
    int i = (int)(xa & 0xff);
    x = int_scaled_f((xa >> 9) & ((1ull << 52) - 1), 0) * z.wf[i];
  } else {
    x = z.Rf + (-log1m_u53_f(xb) / z.Rf);
  }
  return ((xa >> 8) & 1) ? -x : x;
}

// v = 1 + c x > 0 (exact).  FP32: |vf - v| <= |c x| 2^-19.5 + 2^-24.
__device__ __forceinline__ bool mt_v_positive(int xk, u64 xa, u64 xb, const MTParams& p, const ZigDev& z) {
  float cx = p.cf * normal_x_f(xk, xa, xb, z);
  float vf = 1.0f + cx;
  float b = fabsf(cx) * 0x1.0p-17f + 0x1.0p-22f;
  if (vf > b) return true;
  if (vf < -b) return false;
  double x = normal_x_exact(xk, xa, xb, z);
  return __dadd_rn(1.0, __dmul_rn(p.c, x)) > 0.0;
}

// Exact Marsaglia-Tsang test for an accepted normal and uniform word u.  The
// logs are first taken from libm (error below one ulp); the decision stands
// unless the two sides are within the effect of one-ulp log errors, in which
// case the correctly rounded logs decide.
static __device__ bool mt_accept_exact(int xk, u64 xa, u64 xb, u64 u, const MTParams& p, const ZigDev& z) {
  dbg_count(DBG_MT_FP64);
  double x = normal_x_exact(xk, xa, xb, z);
  double v = __dadd_rn(1.0, __dmul_rn(p.c, x));
  v = __dmul_rn(__dmul_rn(v, v), v);
  double U = u53_bits(u);
  double x2 = __dmul_rn(x, x);
  if (U < __dsub_rn(1.0, __dmul_rn(kSqueeze, __dmul_rn(x2, x2)))) return true;
  if (U == 0.0) return true;  // log 0 = -inf
  double om = __dsub_rn(1.0, v);
  double lu = log(U), lv = log(v);
  double s = __dadd_rn(om, lv);
  double ds = __dmul_rn(p.d, s);
  double rhs = __dadd_rn(__dmul_rn(0.5, x2), ds);
  double marg = 0x1.0p-48 * (fabs(lu) + p.d * (fabs(lv) + fabs(s)) + fabs(ds) + fabs(rhs));
  if (lu < rhs - marg) return true;
  if (lu > rhs + marg) return false;
  dbg_count(DBG_MT_CR);
  rhs = __dadd_rn(__dmul_rn(0.5, x2), __dmul_rn(p.d, __dadd_rn(om, cr_log_nl(v))));
  return cr_log_nl(U) < rhs;
}

// Marsaglia-Tsang accept test, FP32 first.  Squeeze: x_f relative 2^-20 so
// 0.0331 x^4 is within q 2^-17.9; margin q 2^-15 + 2^-21.  Log test (only
// with v_f >= 1/4, otherwise exact): v_f is within |c x| 2^-19.5 + 2^-24, so
// (1 - v^3) + log v^3 is within 2^-15.9 absolute for |c x| <= 2 and every
// other term within 2^-19 of its magnitude; the margin is 2^-15 times the sum
// of magnitudes.
__device__ __forceinline__ bool mt_accept(int xk, u64 xa, u64 xb, u64 u, const MTParams& p, const ZigDev& z) {
  float xf = normal_x_f(xk, xa, xb, z);
  float x2f = xf * xf;
  float Uf = u53_f(u);
  float q = 0.0331f * (x2f * x2f);
  float rhs = 1.0f - q;
  float m = q * 0x1.0p-15f + 0x1.0p-21f;
  if (Uf < rhs - m) return true;
  if (Uf > rhs + m) {
    float vf = 1.0f + p.cf * xf;
    if (vf >= 0.25f && (u >> 11) != 0) {
      float v3 = vf * vf * vf;
      float lv = logf(v3);
      float lhs = logf(Uf);
      float r2 = 0.5f * x2f + p.df * ((1.0f - v3) + lv);
      float m2 = 0x1.0p-15f * (1.0f + fabsf(lhs) + 0.5f * x2f + p.df * (1.0f + v3 + fabsf(lv)));
      if (lhs < r2 - m2) return true;
      if (lhs > r2 + m2) return false;
    }
  }
  return mt_accept_exact(xk, xa, xb, u, p, z);
}

// Gamma value of a record (exact FP64, as the serial definition); the boost
// uses the correctly rounded log and libm exp (within 2 ulp).
__device__ __forceinline__ double gamma_value(int xk, u64 xa, u64 xb, u64 ub, const MTParams& p, const ZigDev& z) {
  double x = normal_x_exact(xk, xa, xb, z);
  double v = __dadd_rn(1.0, __dmul_rn(p.c, x));
  v = __dmul_rn(__dmul_rn(v, v), v);
  double g = __dmul_rn(p.d, v);
  if (p.boost) {
    double t = __ddiv_rn(cr_log_nl(u53_bits(ub)), p.alpha);
    g = __dmul_rn(g, exp(t));
  }
  return g;
}

// One gamma chain: the embedded normal candidate parser and the attempt
// states.  feed() returns 1 when a gamma variate is complete; its record is
// (xk, xa, xb) and the boost word ub.
struct GammaMach {
  int ns;   // normal: 0 idle, 1 wedge waiting for U, 2 tail waiting for U1, 3 tail waiting for U2
  int gs;   // attempt: 0 drawing the normal, 1 waiting for U, 2 waiting for the boost word
  int xk;
  u64 nu0, nw1, xa, xb, ub;
  __device__ __forceinline__ void reset() { ns = 0; gs = 0; }
  __device__ __forceinline__ bool idle() const { return ns == 0 && gs == 0; }
  __device__ __forceinline__ int feed(u64 u, const MTParams& p, const ZigDev& z) {
    if (gs == 1) {
      if (!mt_accept(xk, xa, xb, u, p, z)) { gs = 0; return 0; }
      if (p.boost) { gs = 2; return 0; }
      gs = 0;
      ub = 0;
      return 1;
    }
    if (gs == 2) { ub = u; gs = 0; return 1; }
    // normal candidate parsing
    if (ns == 0) {
      int i = (int)(u & 0xff);
      if (((u >> 9) & ((1ull << 52) - 1)) < z.k[i]) {
        xk = 1;
        xa = u;
      } else {
        nu0 = u;
        ns = i ? 1 : 2;
        return 0;
      }
    } else if (ns == 1) {
      ns = 0;
      int i = (int)(nu0 & 0xff);
      if (!wedge_accept<true>((nu0 >> 9) & ((1ull << 52) - 1), i, u, z)) return 0;
      xk = 1;
      xa = nu0;
    } else if (ns == 2) {
      nw1 = u;
      ns = 3;
      return 0;
    } else {
      if (!tail_pair_accept(nw1, u, z)) { ns = 2; return 0; }
      ns = 0;
      xk = 2;
      xa = nu0;
      xb = nw1;
    }
    // an accepted normal x: v = 1 + c x must be positive, else a new attempt
    if (mt_v_positive(xk, xa, xb, p, z)) gs = 1;
    return 0;
  }
};

// One standard normal by the ziggurat, fed word by word: feed() returns 1
// when a normal is accepted; its record is (xk, xa, xb) as in GammaMach.
struct NormalMach {
  int ns;   // 0 idle, 1 wedge waiting for U, 2 tail waiting for U1, 3 tail waiting for U2
  int xk;
  u64 nu0, nw1, xa, xb;
  __device__ __forceinline__ void reset() { ns = 0; }
  __device__ __forceinline__ bool idle() const { return ns == 0; }
  __device__ __forceinline__ int feed(u64 u, const ZigDev& z) {
    if (ns == 0) {
      const int i = (int)(u & 0xff);
      if (((u >> 9) & ((1ull << 52) - 1)) < z.k[i]) { xk = 1; xa = u; return 1; }
      nu0 = u;
      ns = i ? 1 : 2;
      return 0;
    }
    if (ns == 1) {
      ns = 0;
      if (!wedge_accept<true>((nu0 >> 9) & ((1ull << 52) - 1), (int)(nu0 & 0xff), u, z)) return 0;
      xk = 1; xa = nu0;
      return 1;
    }
    if (ns == 2) { nw1 = u; ns = 3; return 0; }
    if (!tail_pair_accept(nw1, u, z)) { ns = 2; return 0; }
    ns = 0;
    xk = 2; xa = nu0; xb = nw1;
    return 1;
  }
};

// Record words of a variate: r[0] = kinds (xk | yk << 8), r[1..3] = X (xa,
// xb, ub), r[4..6] = Y (beta only).
struct SampGamma {
  static constexpr int kChunk = 2048;   // words per thread chunk in a single fill
  static constexpr bool kPhased = false;
  struct M {
    GammaMach g;
    __device__ __forceinline__ void reset() { g.reset(); }
    __device__ __forceinline__ bool idle() const { return g.idle(); }
    __device__ __forceinline__ int feed(u64 u, const SampArgs& a, const ZigDev& z) { return g.feed(u, a.ga, z); }
    __device__ __forceinline__ void record(u64* r) const {
      r[0] = (u64)g.xk;
      r[1] = g.xa; r[2] = g.xb; r[3] = g.ub;
    }
  };
  __device__ static __forceinline__ bool needs_tail(const u64* r) { return (r[0] & 0xff) == 2; }
  __device__ static __forceinline__ double value(const u64* r, const SampArgs& a, const ZigDev& z) {
    const double g = gamma_value((int)(r[0] & 0xff), r[1], r[2], r[3], a.ga, z);
    return a.epi ? epi_value(g, a) : g;   // Gamma(alpha, theta), chi2
  }
};

// Gamma with the boost (alpha < 1): each variate takes longer and its chains
// coalesce more slowly at a seam, so longer chunks pay off, as for beta.
struct SampGammaBoost : SampGamma {
  static constexpr int kChunk = 4096;
};

struct SampBeta {
  // two gamma chains coalesce more slowly at a seam: longer chunks amortise the search
  static constexpr int kChunk = 4096;
  // Seams are phased merge points (merge_tile_ph): a chain's state at a gamma
  // boundary is its phase, 0 (next gamma is X) or 1 (next is Y).
  static constexpr bool kPhased = true;
  // Control state only (no records): the seam searches and the counting walks.
  struct L {
    GammaMach g;
    int ph;
    __device__ __forceinline__ void reset(int p) { g.reset(); ph = p; }
    __device__ __forceinline__ bool idle() const { return g.idle(); }   // at a gamma boundary
    __device__ __forceinline__ int phase() const { return ph; }
    __device__ __forceinline__ int feed(u64 u, const SampArgs& a, const ZigDev& z) {
      if (!g.feed(u, ph ? a.gb : a.ga, z)) return 0;
      ph ^= 1;
      return ph == 0;
    }
  };
  struct M {
    GammaMach g;
    int ph;        // 0 drawing X, 1 drawing Y
    int xk;
    u64 xa, xb, xub;
    __device__ __forceinline__ void reset() { g.reset(); ph = 0; }
    // entering at a gamma boundary in phase p (with p = 1 the first output
    // completes a variate whose X this machine has not seen)
    __device__ __forceinline__ void reset(int p) { g.reset(); ph = p; }
    __device__ __forceinline__ bool idle() const { return g.idle() && ph == 0; }
    __device__ __forceinline__ int feed(u64 u, const SampArgs& a, const ZigDev& z) {
      if (!g.feed(u, ph ? a.gb : a.ga, z)) return 0;
      if (ph == 0) {
        xk = g.xk; xa = g.xa; xb = g.xb; xub = g.ub;
        ph = 1;
        return 0;
      }
      ph = 0;
      return 1;
    }
    __device__ __forceinline__ void record(u64* r) const {
      r[0] = (u64)xk | ((u64)g.xk << 8);
      r[1] = xa; r[2] = xb; r[3] = xub;
      r[4] = g.xa; r[5] = g.xb; r[6] = g.ub;
    }
  };
  __device__ static __forceinline__ bool needs_tail(const u64* r) {
    return (r[0] & 0xff) == 2 || ((r[0] >> 8) & 0xff) == 2;
  }
  __device__ static __forceinline__ double value(const u64* r, const SampArgs& a, const ZigDev& z) {
    double X = gamma_value((int)(r[0] & 0xff), r[1], r[2], r[3], a.ga, z);
    double Y = gamma_value((int)((r[0] >> 8) & 0xff), r[4], r[5], r[6], a.gb, z);
    if (a.epi == EPI_F) return __ddiv_rn(__ddiv_rn(X, a.ep[0]), __ddiv_rn(Y, a.ep[1]));   // F(nu1, nu2)
    return __ddiv_rn(X, __dadd_rn(X, Y));
  }
  // Writes output i, and its gamma pair when the fill keeps them (sp.outx).
  __device__ static __forceinline__ void store(double* out, u64 i, const u64* r, const SampArgs& a, const ZigDev& z) {
    if (!a.outx) {
      out[i] = value(r, a, z);
      return;
    }
    const double X = gamma_value((int)(r[0] & 0xff), r[1], r[2], r[3], a.ga, z);
    const double Y = gamma_value((int)((r[0] >> 8) & 0xff), r[4], r[5], r[6], a.gb, z);
    out[i] = __ddiv_rn(X, __dadd_rn(X, Y));
    a.outx[i] = X;
    a.outy[i] = Y;
  }
};

// Student t (Table "continuous": the normal-gamma mixture Z / sqrt(V / nu)),
// Z ~ N(0, 1) drawn before V ~ chi2_nu = 2 Gamma(nu / 2) from the same
// stream.  Record: r[0] = kinds (Z | V << 8), r[1..2] = Z (xa, xb), r[4..6]
// = the gamma record of V.  ep[0] = nu.
struct SampT {
  static constexpr int kChunk = 4096;   // two sub-variates per output, as beta
  static constexpr bool kPhased = false;
  struct M {
    NormalMach nm;
    GammaMach g;
    int ph;        // 0 drawing Z, 1 drawing V
    __device__ __forceinline__ void reset() { nm.reset(); g.reset(); ph = 0; }
    __device__ __forceinline__ bool idle() const { return ph == 0 && nm.idle(); }
    __device__ __forceinline__ int feed(u64 u, const SampArgs& a, const ZigDev& z) {
      if (ph == 0) {
        if (nm.feed(u, z)) ph = 1;
        return 0;
      }
      if (!g.feed(u, a.ga, z)) return 0;
      ph = 0;
      return 1;
    }
    __device__ __forceinline__ void record(u64* r) const {
      r[0] = (u64)nm.xk | ((u64)g.xk << 8);
      r[1] = nm.xa; r[2] = nm.xb; r[3] = 0;
      r[4] = g.xa; r[5] = g.xb; r[6] = g.ub;
    }
  };
  __device__ static __forceinline__ bool needs_tail(const u64* r) {
    return (r[0] & 0xff) == 2 || ((r[0] >> 8) & 0xff) == 2;
  }
  __device__ static __forceinline__ double value(const u64* r, const SampArgs& a, const ZigDev& z) {
    const double Z = normal_x_exact((int)(r[0] & 0xff), r[1], r[2], z);
    const double V = __dmul_rn(2.0, gamma_value((int)((r[0] >> 8) & 0xff), r[4], r[5], r[6], a.ga, z));
    return __ddiv_rn(Z, __dsqrt_rn(__ddiv_rn(V, a.ep[0])));
  }
};
