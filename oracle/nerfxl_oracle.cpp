// NeRF-XL CPU oracle (arXiv 2404.16221) -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct statement of what the one-GPU hot path
// computes, in FP64 (plus the prescribed FP32 geometry/index path below).
// Only the test suite, the package smoke check and the CPU-baseline leg of the
// benchmark may load this library. It shares no code, header, table or
// constant generator with the CUDA path; the two meet only through the seeded
// synthetic inputs both are handed.
//
// What each part follows:
//   * Volume rendering integral and its piecewise-constant discretisation:
//     Sec. 4.1, Eq. 1. Each interval carries one density and one colour, so the
//     per-interval integral is exact: T_i * (1 - exp(-sigma_i delta_i)) * c_i.
//   * Distortion loss: Sec. 4.1, Eq. 2, in raw ray distance t, each interval's
//     weight spread uniformly over it (the Mip-NeRF 360 step-function form):
//         L = sum_{i,j} w_i w_j |tbar_i - tbar_j| + 1/3 sum_i w_i^2 delta_i.
//   * Non-overlapping tiles, samples assigned by box, no interval crossing a
//     box face: Sec. 4.2.
//   * Partitioned rendering (per-segment partials, then exclusive prefix
//     product in ray order): Sec. 4.3, Eq. 3-8, Algorithm 1 and Algorithm 2.
//     Two readings: the cross term of Algorithm 2 uses the s-th segment's own
//     D and A (as Eq. 8 writes it), and it carries the factor 2 of Eq. 7.
//   * Per-tile Instant-NGP field: Appendix A.1 (the hash encoding is the one
//     defined by the cited Instant-NGP paper: dense index where (N+1)^3 <= T,
//     else XOR of coordinates times the primes 1, 2654435761, 805459861,
//     modulo T), followed by a ReLU MLP without biases, density = exp(o0),
//     colour = sigmoid(o1..o3).
//   * Loss: mean squared RGB error + lambda * mean distortion; Adam (Kingma &
//     Ba) with bias correction.
//   * Split representation (App. A.1, the representation the paper trains):
//     per region a hash encoding and a density MLP with one hidden layer,
//     feat -> 64 -> 16 (ReLU, no biases), density = exp(g0); one colour MLP
//     shared by all regions on [g (16), SH(d) (16)] -> 64 -> 64 -> 3, colour =
//     sigmoid. The view direction is encoded by the real spherical harmonics
//     of degrees 0-3 (Instant-NGP's direction encoding), written out below
//     from their Cartesian closed forms. No appearance embedding (it is zero
//     at novel-view rendering and there are no per-image captures here).
//   * Occupancy grid (the spatial-skipping structure every compared method
//     uses, Sec. 5.1; the grid is the one of the cited Instant-NGP paper): per
//     region a G^3 grid of cells over the region box, one bit each. A sample
//     whose point falls in a cell with a clear bit is rendered with density 0
//     (it is not evaluated, and no gradient flows through it). The grid is
//     refreshed from the field: each cell's density estimate becomes
//     max(decay * old, sigma(p)) at one point p drawn uniformly in the cell,
//     and its bit is set where the estimate exceeds a threshold. The points
//     come from Philox4x32-10 (Salmon et al., SC 2011), written out below from
//     its published definition.
//   * Test diagnostics, not part of the method: the distance of each sample's
//     hidden units from their ReLU kinks relative to their rounding-error
//     scale (which rays an FP32 gradient may legitimately see on the other
//     side of a kink), and the pinhole rays of a render request in a
//     prescribed FP32 operation order (the rays a served image is checked on).
//
// Parity status: every function here is pinned by CPU tests (closed forms,
// brute force, library GEMMs, finite differences); none is "parity unpinned".
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math -shared -fPIC -pthread

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

typedef struct {
  int32_t K, L, F, log2_T, mlp_in, W;
  const int32_t* level_res;  // [L]  grid resolution N_l of each level
  const float* boxes;        // [K][6] min xyz, max xyz (disjoint)
  const double* tables;      // [K][E][F]  E = sum of level sizes
  const double* mlp;         // [K][P]  W1[mlp_in][W] W2[W][W] W3[W][4]
  const uint32_t* occupancy; // [K][ceil(G^3/32)] cell bits, or NULL (no skipping)
  int32_t occ_res;           // G: cells per axis of each region's grid
  int32_t arch;              // 0: one MLP per region; 1: density MLP per region + shared colour MLP
} oracle_field;

typedef struct {
  int32_t S;      // uniform grid intervals over [first t0, last t1]
  float t_min;    // near clamp (0)
} oracle_sampling;

}  // extern "C"

namespace {

const uint32_t kPrime2 = 2654435761u;  // Instant-NGP spatial hash primes
const uint32_t kPrime3 = 805459861u;

int g_threads = 0;

int n_threads() {
  if (g_threads > 0) return g_threads;
  unsigned h = std::thread::hardware_concurrency();
  return h == 0 ? 1 : (int)h;
}

// Runs fn(r, thread) for r in [0, n) over a pool of plain threads.
template <class Fn>
void parallel_for(int64_t n, Fn fn) {
  int nt = n_threads();
  if (nt <= 1 || n < 32) {
    for (int64_t r = 0; r < n; ++r) fn(r, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) {
    pool.emplace_back([&, t]() {
      for (;;) {
        int64_t r0 = next.fetch_add(8);
        if (r0 >= n) break;
        int64_t r1 = std::min(n, r0 + 8);
        for (int64_t r = r0; r < r1; ++r) fn(r, t);
      }
    });
  }
  for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------
// Level layout: level l has N_l cells per axis and (N_l+1)^3 lattice vertices.
// If (N_l+1)^3 <= T it is stored densely ((N_l+1)^3 entries, rounded up to a
// multiple of 8), else it holds T hashed entries.
struct Level {
  int32_t N;
  bool dense;
  int64_t offset;  // in entries, within one region's table
  int64_t size;
};

std::vector<Level> make_levels(int L, const int32_t* res, int log2_T) {
  std::vector<Level> lv(L);
  const int64_t T = int64_t(1) << log2_T;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    const int64_t v = int64_t(res[l]) + 1;
    const int64_t verts = v * v * v;
    lv[l].N = res[l];
    lv[l].dense = verts <= T;
    lv[l].size = lv[l].dense ? ((verts + 7) / 8) * 8 : T;
    lv[l].offset = off;
    off += lv[l].size;
  }
  return lv;
}

int64_t mlp_params(int mlp_in, int W) { return int64_t(mlp_in) * W + int64_t(W) * W + int64_t(W) * 4; }

// Split representation: density block Wd1 [mlp_in][W], Wd2 [W][16] per region;
// shared colour block Wc1 [32][W], Wc2 [W][W], Wc3 [W][4] (column 3 unused).
const int kGeo = 16;  // density MLP outputs: g0 (log density) and 15 more geometry features
const int kSh = 16;   // spherical-harmonic coefficients of degrees 0..3
int64_t density_params(int mlp_in, int W) { return int64_t(mlp_in) * W + int64_t(W) * kGeo; }
int64_t color_params(int W) { return int64_t(kGeo + kSh) * W + int64_t(W) * W + int64_t(W) * 4; }
// Elements of the field's mlp array.
int64_t field_mlp_size(const oracle_field& f) {
  return f.arch == 1 ? int64_t(f.K) * density_params(f.mlp_in, f.W) + color_params(f.W)
                     : int64_t(f.K) * mlp_params(f.mlp_in, f.W);
}

// Real spherical harmonics of degrees 0..3 at the unit vector (x, y, z), with
// the Condon-Shortley phase: Y_l^m for m = -l..l, degree by degree. Each
// constant is the normalisation sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times
// sqrt 2 for m != 0) folded with the Cartesian form of its associated
// Legendre factor.
void sh4(const double* d, double* y) {
  const double x = d[0], yy = d[1], z = d[2];
  const double pi = 3.14159265358979323846;
  const double c0 = 0.5 * std::sqrt(1.0 / pi);
  const double c1 = std::sqrt(3.0 / (4.0 * pi));
  const double c2a = 0.5 * std::sqrt(15.0 / pi), c2b = 0.25 * std::sqrt(5.0 / pi), c2c = 0.25 * std::sqrt(15.0 / pi);
  const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * pi)), c3b = 0.5 * std::sqrt(105.0 / pi);
  const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * pi)), c3d = 0.25 * std::sqrt(7.0 / pi);
  const double c3e = 0.25 * std::sqrt(105.0 / pi);
  y[0] = c0;
  y[1] = -c1 * yy;
  y[2] = c1 * z;
  y[3] = -c1 * x;
  y[4] = c2a * x * yy;
  y[5] = -c2a * yy * z;
  y[6] = c2b * (3.0 * z * z - 1.0);
  y[7] = -c2a * x * z;
  y[8] = c2c * (x * x - yy * yy);
  y[9] = -c3a * yy * (3.0 * x * x - yy * yy);
  y[10] = c3b * x * yy * z;
  y[11] = -c3c * yy * (5.0 * z * z - 1.0);
  y[12] = c3d * z * (5.0 * z * z - 3.0);
  y[13] = -c3c * x * (5.0 * z * z - 1.0);
  y[14] = c3e * z * (x * x - yy * yy);
  y[15] = -c3a * x * (x * x - 3.0 * yy * yy);
}

// ---------------------------------------------------------------------------
// Geometry, in the prescribed FP32 operation order (one IEEE rounding per op).
struct Seg {
  int region;
  float t0, t1;
};
struct Interval {
  float a, b;
  int region;
  int seg;  // index of its segment within the ray
};

// Slab test of one ray against one box; NaN-ignoring min/max (fmin/fmax).
bool slab(const float* o, const float* d, const float* box, float t_min, float* t0, float* t1) {
  float tn = -INFINITY, tf = INFINITY;
  for (int ax = 0; ax < 3; ++ax) {
    const float inv = 1.0f / d[ax];
    const float ta = (box[ax] - o[ax]) * inv;
    const float tb = (box[3 + ax] - o[ax]) * inv;
    tn = std::fmax(tn, std::fmin(ta, tb));
    tf = std::fmin(tf, std::fmax(ta, tb));
  }
  tn = std::fmax(tn, t_min);
  *t0 = tn;
  *t1 = tf;
  return tf > tn;
}

// Sec. 4.2: the ray's box segments in ray order (sorted by t0, then region id).
std::vector<Seg> ray_segments(const oracle_field& f, const oracle_sampling& s, const float* o, const float* d) {
  std::vector<Seg> segs;
  for (int k = 0; k < f.K; ++k) {
    float t0, t1;
    if (slab(o, d, f.boxes + 6 * k, s.t_min, &t0, &t1)) segs.push_back({k, t0, t1});
  }
  std::sort(segs.begin(), segs.end(), [](const Seg& x, const Seg& y) {
    if (x.t0 != y.t0) return x.t0 < y.t0;
    return x.region < y.region;
  });
  return segs;
}

// Uniform grid of S intervals over [first t0, last t1], cut at every segment
// end: segment k owns the edges {t0_k} U {e_j : t0_k < e_j < t1_k} U {t1_k}.
// e_j = tn + j * ((tf - tn) / S), j = 1..S-1, each op rounded in FP32.
std::vector<Interval> ray_intervals(const std::vector<Seg>& segs, int S) {
  std::vector<Interval> iv;
  if (segs.empty()) return iv;
  const float tn = segs.front().t0;
  const float tf = segs.back().t1;
  const float delta = (tf - tn) / (float)S;
  for (size_t k = 0; k < segs.size(); ++k) {
    std::vector<float> edges;
    edges.push_back(segs[k].t0);
    for (int j = 1; j < S; ++j) {
      const float e = tn + (float)j * delta;
      if (e > segs[k].t0 && e < segs[k].t1) edges.push_back(e);
    }
    edges.push_back(segs[k].t1);
    for (size_t i = 0; i + 1 < edges.size(); ++i) iv.push_back({edges[i], edges[i + 1], segs[k].region, (int)k});
  }
  return iv;
}

// ---------------------------------------------------------------------------
// Hash-grid encoding of one point of one region (Instant-NGP, cited by App. A.1).
struct Encoded {
  std::vector<double> feat;        // [mlp_in], zero beyond L*F
  std::vector<int64_t> entry;      // [L][8] entry index within the region table
  std::vector<double> weight;      // [L][8] trilinear weight
  std::vector<uint32_t> index;     // [L][8] index within the level
};

// Region-local coordinate u = clamp((x - bmin) / (bmax - bmin), 0, 1), with
// the reciprocal of the extent taken first (FP32).
void region_u(const float* box, const float* x, float* u) {
  for (int ax = 0; ax < 3; ++ax) {
    const float inv_ext = 1.0f / (box[3 + ax] - box[ax]);
    float v = (x[ax] - box[ax]) * inv_ext;
    v = std::fmin(std::fmax(v, 0.0f), 1.0f);
    u[ax] = v;
  }
}

// Cell of region coordinate u in a grid of N cells per axis: min(floor(u N), N - 1).
int32_t grid_cell(float u, int32_t N) {
  const float p = u * (float)N;
  int32_t c = (int32_t)std::floor(p);
  if (c > N - 1) c = N - 1;
  if (c < 0) c = 0;
  return c;
}

void encode_u(const oracle_field& f, const std::vector<Level>& lv, int region, const float* u, Encoded* out);

void encode(const oracle_field& f, const std::vector<Level>& lv, int region, const float* x, Encoded* out) {
  float u[3];
  region_u(f.boxes + 6 * region, x, u);
  encode_u(f, lv, region, u, out);
}

// Encoding at region coordinate u.
void encode_u(const oracle_field& f, const std::vector<Level>& lv, int region, const float* u, Encoded* out) {
  const int64_t E = lv.back().offset + lv.back().size;
  const double* table = f.tables + int64_t(region) * E * f.F;
  const uint32_t T = uint32_t(1) << f.log2_T;
  out->feat.assign(f.mlp_in, 0.0);
  out->entry.assign(f.L * 8, 0);
  out->weight.assign(f.L * 8, 0.0);
  out->index.assign(f.L * 8, 0);
  for (int l = 0; l < f.L; ++l) {
    const int32_t N = lv[l].N;
    int32_t c[3];
    float fr[3];
    for (int ax = 0; ax < 3; ++ax) {
      const float p = u[ax] * (float)N;
      int32_t ci = (int32_t)std::floor(p);
      if (ci > N - 1) ci = N - 1;
      if (ci < 0) ci = 0;
      c[ax] = ci;
      fr[ax] = p - (float)ci;
    }
    for (int e = 0; e < 8; ++e) {
      const uint32_t vx = uint32_t(c[0] + (e & 1));
      const uint32_t vy = uint32_t(c[1] + ((e >> 1) & 1));
      const uint32_t vz = uint32_t(c[2] + ((e >> 2) & 1));
      uint32_t idx;
      if (lv[l].dense) {
        const uint32_t side = uint32_t(N) + 1;
        idx = vx + vy * side + vz * side * side;
      } else {
        idx = ((vx * 1u) ^ (vy * kPrime2) ^ (vz * kPrime3)) & (T - 1);
      }
      double w = 1.0;
      for (int ax = 0; ax < 3; ++ax) {
        const int bit = (e >> ax) & 1;
        w *= bit ? (double)fr[ax] : (1.0 - (double)fr[ax]);
      }
      const int64_t entry = lv[l].offset + idx;
      out->index[l * 8 + e] = idx;
      out->entry[l * 8 + e] = entry;
      out->weight[l * 8 + e] = w;
      for (int j = 0; j < f.F; ++j) out->feat[l * f.F + j] += w * table[entry * f.F + j];
    }
  }
}

// ---------------------------------------------------------------------------
// MLP: z1 = W1^T feat, h1 = relu(z1), z2 = W2^T h1, h2 = relu(z2), o = W3^T h2.
// Split representation: z1 = Wd1^T feat, h1 = relu(z1), g = Wd2^T h1 (o0 = g0);
// xc = [g, SH(d)], z2 = Wc1^T xc, h2 = relu(z2), z3 = Wc2^T h2, h3 = relu(z3),
// o1..3 = Wc3^T h3.
struct MlpAct {
  std::vector<double> z1, h1, z2, h2;
  std::vector<double> xc, z3, h3;  // split representation only
  double o[4];
};

void mlp_forward_split(const oracle_field& f, int region, const double* feat, const float* dir, MlpAct* a) {
  const int W = f.W, I = f.mlp_in;
  const double* Wd1 = f.mlp + int64_t(region) * density_params(I, W);
  const double* Wd2 = Wd1 + int64_t(I) * W;
  const double* Wc1 = f.mlp + int64_t(f.K) * density_params(I, W);
  const double* Wc2 = Wc1 + int64_t(kGeo + kSh) * W;
  const double* Wc3 = Wc2 + int64_t(W) * W;
  a->z1.assign(W, 0.0);
  a->h1.assign(W, 0.0);
  for (int n = 0; n < W; ++n) {
    double s = 0.0;
    for (int i = 0; i < I; ++i) s += feat[i] * Wd1[i * W + n];
    a->z1[n] = s;
    a->h1[n] = s > 0.0 ? s : 0.0;
  }
  a->xc.assign(kGeo + kSh, 0.0);
  for (int m = 0; m < kGeo; ++m) {
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += a->h1[i] * Wd2[i * kGeo + m];
    a->xc[m] = s;
  }
  const double dd[3] = {(double)dir[0], (double)dir[1], (double)dir[2]};
  sh4(dd, a->xc.data() + kGeo);
  a->z2.assign(W, 0.0);
  a->h2.assign(W, 0.0);
  for (int n = 0; n < W; ++n) {
    double s = 0.0;
    for (int i = 0; i < kGeo + kSh; ++i) s += a->xc[i] * Wc1[i * W + n];
    a->z2[n] = s;
    a->h2[n] = s > 0.0 ? s : 0.0;
  }
  a->z3.assign(W, 0.0);
  a->h3.assign(W, 0.0);
  for (int n = 0; n < W; ++n) {
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += a->h2[i] * Wc2[i * W + n];
    a->z3[n] = s;
    a->h3[n] = s > 0.0 ? s : 0.0;
  }
  a->o[0] = a->xc[0];
  for (int m = 0; m < 3; ++m) {
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += a->h3[i] * Wc3[i * 4 + m];
    a->o[1 + m] = s;
  }
}

void mlp_forward(const oracle_field& f, int region, const double* feat, const float* dir, MlpAct* a) {
  if (f.arch == 1) {
    mlp_forward_split(f, region, feat, dir, a);
    return;
  }
  const int W = f.W, I = f.mlp_in;
  const double* p = f.mlp + int64_t(region) * mlp_params(I, W);
  const double* W1 = p;
  const double* W2 = W1 + int64_t(I) * W;
  const double* W3 = W2 + int64_t(W) * W;
  a->z1.assign(W, 0.0);
  a->h1.assign(W, 0.0);
  a->z2.assign(W, 0.0);
  a->h2.assign(W, 0.0);
  for (int n = 0; n < W; ++n) {
    double s = 0.0;
    for (int i = 0; i < I; ++i) s += feat[i] * W1[i * W + n];
    a->z1[n] = s;
    a->h1[n] = s > 0.0 ? s : 0.0;
  }
  for (int n = 0; n < W; ++n) {
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += a->h1[i] * W2[i * W + n];
    a->z2[n] = s;
    a->h2[n] = s > 0.0 ? s : 0.0;
  }
  for (int m = 0; m < 4; ++m) {
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += a->h2[i] * W3[i * 4 + m];
    a->o[m] = s;
  }
}

double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }

// ---------------------------------------------------------------------------
// One ray's samples, with the field evaluated at every interval midpoint.
struct RayEval {
  std::vector<Interval> iv;
  std::vector<double> tbar, delta, sigma;
  std::vector<double> rgb;  // [n][3]
  std::vector<Encoded> enc;
  std::vector<MlpAct> act;
  std::vector<char> skip;   // 1: the sample's occupancy cell is empty (density 0, not evaluated)
};

// Occupancy bit of the cell holding region coordinate u (1 without a grid).
bool occupied(const oracle_field& f, int region, const float* u) {
  if (!f.occupancy) return true;
  const int64_t G = f.occ_res;
  const int64_t words = (G * G * G + 31) / 32;
  const int64_t cell = grid_cell(u[0], f.occ_res) + G * (grid_cell(u[1], f.occ_res) + G * grid_cell(u[2], f.occ_res));
  return ((f.occupancy[int64_t(region) * words + cell / 32] >> (cell % 32)) & 1u) != 0;
}

void eval_ray(const oracle_field& f, const oracle_sampling& s, const std::vector<Level>& lv, const float* o,
              const float* d, bool keep, RayEval* re) {
  re->iv = ray_intervals(ray_segments(f, s, o, d), s.S);
  const size_t n = re->iv.size();
  re->tbar.resize(n);
  re->delta.resize(n);
  re->sigma.resize(n);
  re->rgb.resize(3 * n);
  re->skip.assign(n, 0);
  if (keep) {
    re->enc.resize(n);
    re->act.resize(n);
  }
  Encoded enc;
  MlpAct act;
  for (size_t i = 0; i < n; ++i) {
    const Interval& q = re->iv[i];
    const float tb = 0.5f * (q.a + q.b);
    const float dl = q.b - q.a;
    float x[3];
    for (int ax = 0; ax < 3; ++ax) x[ax] = o[ax] + tb * d[ax];
    re->tbar[i] = tb;
    re->delta[i] = dl;
    float u[3];
    region_u(f.boxes + 6 * q.region, x, u);
    if (!occupied(f, q.region, u)) {
      re->skip[i] = 1;
      re->sigma[i] = 0.0;
      for (int c = 0; c < 3; ++c) re->rgb[3 * i + c] = 0.0;
      continue;
    }
    encode(f, lv, q.region, x, &enc);
    mlp_forward(f, q.region, enc.feat.data(), d, &act);
    re->sigma[i] = std::exp(act.o[0]);
    for (int c = 0; c < 3; ++c) re->rgb[3 * i + c] = sigmoid(act.o[1 + c]);
    if (keep) {
      re->enc[i] = enc;
      re->act[i] = act;
    }
  }
}

// ---------------------------------------------------------------------------
// Rendering of explicit per-interval values.
// out[0..2] = C, out[3] = D, out[4] = A, out[5] = L_dist, out[6] = T_final.

// (i) Single pass over all intervals (Eq. 1, Eq. 2 written out; O(N^2) distortion).
void render_single(size_t n, const double* sigma, const double* rgb, const double* tbar, const double* delta,
                   double* out) {
  std::vector<double> w(n);
  double acc = 0.0;
  double C[3] = {0, 0, 0}, A = 0, D = 0;
  for (size_t i = 0; i < n; ++i) {
    const double tau = sigma[i] * delta[i];
    const double T = std::exp(-acc);
    w[i] = T * -std::expm1(-tau);
    for (int c = 0; c < 3; ++c) C[c] += w[i] * rgb[3 * i + c];
    A += w[i];
    D += w[i] * tbar[i];
    acc += tau;
  }
  double Ld = 0.0;
  for (size_t i = 0; i < n; ++i) {
    for (size_t j = 0; j < n; ++j) Ld += w[i] * w[j] * std::fabs(tbar[i] - tbar[j]);
    Ld += w[i] * w[i] * delta[i] / 3.0;
  }
  out[0] = C[0];
  out[1] = C[1];
  out[2] = C[2];
  out[3] = D;
  out[4] = A;
  out[5] = Ld;
  out[6] = std::exp(-acc);
}

// Segment-local rendering (transmittance restarts at 1 inside the segment):
// part = {tau_k, C_k[3], A_k, D_k, L_k}, L_k by the O(n) prefix-sum form
// L_k = sum_i [ 2 w_i (tbar_i W_<i - WT_<i) + w_i^2 delta_i / 3 ].
void render_local(size_t n, const double* sigma, const double* rgb, const double* tbar, const double* delta,
                  double* part) {
  double acc = 0.0, C[3] = {0, 0, 0}, A = 0, D = 0, Ld = 0, Wp = 0, WTp = 0;
  for (size_t i = 0; i < n; ++i) {
    const double tau = sigma[i] * delta[i];
    const double w = std::exp(-acc) * -std::expm1(-tau);
    for (int c = 0; c < 3; ++c) C[c] += w * rgb[3 * i + c];
    A += w;
    D += w * tbar[i];
    Ld += 2.0 * w * (tbar[i] * Wp - WTp) + w * w * delta[i] / 3.0;
    Wp += w;
    WTp += w * tbar[i];
    acc += tau;
  }
  part[0] = acc;
  part[1] = C[0];
  part[2] = C[1];
  part[3] = C[2];
  part[4] = A;
  part[5] = D;
  part[6] = Ld;
}

// (ii) Algorithm 1 + Algorithm 2: composite segment partials in ray order.
// T (prefix transmittance) starts at 1; A, D, L, C start at 0; for each
// segment: L += T^2 L_s + 2 T (D_s A - A_s D); C += T C_s; A += T A_s;
// D += T D_s; T *= exp(-tau_s).
void composite(size_t nseg, const double* parts, double* out) {
  double T = 1.0, C[3] = {0, 0, 0}, A = 0, D = 0, Ld = 0;
  for (size_t s = 0; s < nseg; ++s) {
    const double* p = parts + 7 * s;
    const double S = p[5] * A - p[4] * D;
    Ld += T * T * p[6] + 2.0 * T * S;
    for (int c = 0; c < 3; ++c) C[c] += T * p[1 + c];
    A += T * p[4];
    D += T * p[5];
    T *= std::exp(-p[0]);
  }
  out[0] = C[0];
  out[1] = C[1];
  out[2] = C[2];
  out[3] = D;
  out[4] = A;
  out[5] = Ld;
  out[6] = T;
}

void render_partitioned(size_t n, const int* seg_of, const double* sigma, const double* rgb, const double* tbar,
                        const double* delta, double* out) {
  std::vector<double> parts;
  size_t i = 0;
  while (i < n) {
    size_t j = i;
    while (j < n && seg_of[j] == seg_of[i]) ++j;
    double p[7];
    render_local(j - i, sigma + i, rgb + 3 * i, tbar + i, delta + i, p);
    parts.insert(parts.end(), p, p + 7);
    i = j;
  }
  composite(parts.size() / 7, parts.data(), out);
}

void render_ray(const RayEval& re, int mode, double* out) {
  const size_t n = re.iv.size();
  if (mode == 0) {
    render_single(n, re.sigma.data(), re.rgb.data(), re.tbar.data(), re.delta.data(), out);
  } else {
    std::vector<int> seg_of(n);
    for (size_t i = 0; i < n; ++i) seg_of[i] = re.iv[i].seg;
    render_partitioned(n, seg_of.data(), re.sigma.data(), re.rgb.data(), re.tbar.data(), re.delta.data(), out);
  }
}

// ---------------------------------------------------------------------------
// Reverse mode of the single-pass render of one ray, given adjoints of the
// outputs gC[3], gD, gA, gL. Using w_i = T_i - T_{i+1}:
//   dw_j/dtau_i = T_{i+1} if j == i, -w_j if j > i, 0 if j < i,
// so  g_tau_i = g_w_i T_{i+1} - sum_{j>i} g_w_j w_j, with
//   g_w_i = gC.c_i + gA + gD tbar_i + gL (2 sum_j w_j |tbar_i - tbar_j| + 2/3 w_i delta_i).
void render_single_adjoint(size_t n, const double* sigma, const double* rgb, const double* tbar,
                           const double* delta, const double* gC, double gD, double gA, double gL,
                           double* g_sigma, double* g_rgb) {
  std::vector<double> w(n), Tnext(n), gw(n);
  double acc = 0.0;
  for (size_t i = 0; i < n; ++i) {
    const double tau = sigma[i] * delta[i];
    w[i] = std::exp(-acc) * -std::expm1(-tau);
    acc += tau;
    Tnext[i] = std::exp(-acc);
  }
  for (size_t i = 0; i < n; ++i) {
    double pair = 0.0;
    for (size_t j = 0; j < n; ++j) pair += w[j] * std::fabs(tbar[i] - tbar[j]);
    gw[i] = gC[0] * rgb[3 * i] + gC[1] * rgb[3 * i + 1] + gC[2] * rgb[3 * i + 2] + gA + gD * tbar[i] +
            gL * (2.0 * pair + 2.0 / 3.0 * w[i] * delta[i]);
  }
  for (size_t i = 0; i < n; ++i) {
    double later = 0.0;
    for (size_t j = i + 1; j < n; ++j) later += gw[j] * w[j];
    const double g_tau = gw[i] * Tnext[i] - later;
    g_sigma[i] = g_tau * delta[i];
    for (int c = 0; c < 3; ++c) g_rgb[3 * i + c] = w[i] * gC[c];
  }
}

struct Grads {
  std::vector<double> mlp;                          // dense [K][P]
  std::vector<std::pair<int64_t, double>> table;    // (flat index into [K][E][F], value)
};

// Adjoint of field evaluation for one ray: MLP reverse mode then the
// trilinear scatter into the table entries that were read.
// Reverse mode through the split representation for one sample: go[0] is
// dL/dg0 (the log density), go[1..3] dL/d(colour logits). Accumulates into the
// region's density block and the shared colour block of gm; returns dL/dfeat.
void mlp_adjoint_split(const oracle_field& f, int k, const MlpAct& a, const double* feat, const double* go,
                       double* gm, double* gfeat) {
  const int W = f.W, I = f.mlp_in;
  const int64_t Pd = density_params(I, W);
  const double* Wd1 = f.mlp + int64_t(k) * Pd;
  const double* Wd2 = Wd1 + int64_t(I) * W;
  const double* Wc1 = f.mlp + int64_t(f.K) * Pd;
  const double* Wc2 = Wc1 + int64_t(kGeo + kSh) * W;
  const double* Wc3 = Wc2 + int64_t(W) * W;
  double* gd1 = gm + int64_t(k) * Pd;
  double* gd2 = gd1 + int64_t(I) * W;
  double* gc1 = gm + int64_t(f.K) * Pd;
  double* gc2 = gc1 + int64_t(kGeo + kSh) * W;
  double* gc3 = gc2 + int64_t(W) * W;
  std::vector<double> gz3(W), gz2(W), gxc(kGeo + kSh), gz1(W);
  for (int n = 0; n < W; ++n) {  // colour output layer
    double s = 0.0;
    for (int m = 0; m < 3; ++m) {
      gc3[n * 4 + m] += a.h3[n] * go[1 + m];
      s += Wc3[n * 4 + m] * go[1 + m];
    }
    gz3[n] = a.z3[n] > 0.0 ? s : 0.0;
  }
  for (int r = 0; r < W; ++r) {
    double s = 0.0;
    for (int n = 0; n < W; ++n) {
      gc2[r * W + n] += a.h2[r] * gz3[n];
      s += Wc2[r * W + n] * gz3[n];
    }
    gz2[r] = a.z2[r] > 0.0 ? s : 0.0;
  }
  for (int r = 0; r < kGeo + kSh; ++r) {
    double s = 0.0;
    for (int n = 0; n < W; ++n) {
      gc1[r * W + n] += a.xc[r] * gz2[n];
      s += Wc1[r * W + n] * gz2[n];
    }
    gxc[r] = s;  // the direction part (r >= kGeo) has no parameters behind it
  }
  gxc[0] += go[0];  // g0 feeds the density as well as the colour MLP
  for (int r = 0; r < W; ++r) {
    double s = 0.0;
    for (int m = 0; m < kGeo; ++m) {
      gd2[r * kGeo + m] += a.h1[r] * gxc[m];
      s += Wd2[r * kGeo + m] * gxc[m];
    }
    gz1[r] = a.z1[r] > 0.0 ? s : 0.0;
  }
  for (int r = 0; r < I; ++r) {
    double s = 0.0;
    for (int n = 0; n < W; ++n) {
      gd1[r * W + n] += feat[r] * gz1[n];
      s += Wd1[r * W + n] * gz1[n];
    }
    gfeat[r] = s;
  }
}

// Adjoint of field evaluation for one ray: MLP reverse mode then the
// trilinear scatter into the table entries that were read.
void field_adjoint(const oracle_field& f, const RayEval& re, const double* g_sigma, const double* g_rgb,
                   int64_t E, Grads* g) {
  const int W = f.W, I = f.mlp_in;
  const int64_t P = mlp_params(I, W);
  std::vector<double> gz2(W), gz1(W), gfeat(I);
  for (size_t i = 0; i < re.iv.size(); ++i) {
    if (re.skip[i]) continue;  // density fixed at 0: no parameter reaches it
    const int k = re.iv[i].region;
    const MlpAct& a = re.act[i];
    const Encoded& e = re.enc[i];
    double go[4];
    go[0] = g_sigma[i] * re.sigma[i];
    for (int c = 0; c < 3; ++c) {
      const double cc = re.rgb[3 * i + c];
      go[1 + c] = g_rgb[3 * i + c] * cc * (1.0 - cc);
    }
    if (f.arch == 1) {
      mlp_adjoint_split(f, k, a, e.feat.data(), go, g->mlp.data(), gfeat.data());
    } else {
      const double* p = f.mlp + int64_t(k) * P;
      const double* W1 = p;
      const double* W2 = W1 + int64_t(I) * W;
      const double* W3 = W2 + int64_t(W) * W;
      double* g1 = g->mlp.data() + int64_t(k) * P;
      double* g2 = g1 + int64_t(I) * W;
      double* g3 = g2 + int64_t(W) * W;
      for (int n = 0; n < W; ++n) {
        double s = 0.0;
        for (int m = 0; m < 4; ++m) {
          g3[n * 4 + m] += a.h2[n] * go[m];
          s += W3[n * 4 + m] * go[m];
        }
        gz2[n] = a.z2[n] > 0.0 ? s : 0.0;
      }
      for (int r = 0; r < W; ++r) {
        double s = 0.0;
        for (int n = 0; n < W; ++n) {
          g2[r * W + n] += a.h1[r] * gz2[n];
          s += W2[r * W + n] * gz2[n];
        }
        gz1[r] = a.z1[r] > 0.0 ? s : 0.0;
      }
      for (int r = 0; r < I; ++r) {
        double s = 0.0;
        for (int n = 0; n < W; ++n) {
          g1[r * W + n] += e.feat[r] * gz1[n];
          s += W1[r * W + n] * gz1[n];
        }
        gfeat[r] = s;
      }
    }
    for (int l = 0; l < f.L; ++l) {
      for (int c = 0; c < 8; ++c) {
        const int64_t base = (int64_t(k) * E + e.entry[l * 8 + c]) * f.F;
        for (int j = 0; j < f.F; ++j) g->table.push_back({base + j, e.weight[l * 8 + c] * gfeat[l * f.F + j]});
      }
    }
  }
}

// Shared driver of the adjoint: per ray upstream adjoints, dense outputs.
// Per-ray contributions are reduced in ray order, so the result is
// reproducible run to run.
void render_grad_impl(const oracle_field& f, const oracle_sampling& s, int64_t R, const float* ro, const float* rd,
                      const double* gC, const double* gD, const double* gA, const double* gL, double* g_tables,
                      double* g_mlp) {
  const std::vector<Level> lv = make_levels(f.L, f.level_res, f.log2_T);
  const int64_t E = lv.back().offset + lv.back().size;
  std::vector<Grads> per_ray(R);
  parallel_for(R, [&](int64_t r, int) {
    RayEval re;
    eval_ray(f, s, lv, ro + 3 * r, rd + 3 * r, true, &re);
    const size_t n = re.iv.size();
    std::vector<double> gs(n), gc(3 * n);
    render_single_adjoint(n, re.sigma.data(), re.rgb.data(), re.tbar.data(), re.delta.data(), gC + 3 * r, gD[r],
                          gA[r], gL[r], gs.data(), gc.data());
    // MLP gradient of this ray: only the regions it touches are non-zero.
    Grads g;
    g.mlp.assign(size_t(field_mlp_size(f)), 0.0);
    field_adjoint(f, re, gs.data(), gc.data(), E, &g);
    per_ray[r] = std::move(g);
  });
  for (int64_t r = 0; r < R; ++r) {
    for (auto& kv : per_ray[r].table) g_tables[kv.first] += kv.second;
    for (size_t i = 0; i < per_ray[r].mlp.size(); ++i) g_mlp[i] += per_ray[r].mlp[i];
    per_ray[r] = Grads();
  }
}

double loss_impl(const oracle_field& f, const oracle_sampling& s, int64_t R, const float* ro, const float* rd,
                 const float* target, double lambda) {
  const std::vector<Level> lv = make_levels(f.L, f.level_res, f.log2_T);
  std::vector<double> photo(R), dist(R);
  parallel_for(R, [&](int64_t r, int) {
    RayEval re;
    eval_ray(f, s, lv, ro + 3 * r, rd + 3 * r, false, &re);
    double out[7];
    render_ray(re, 0, out);
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double diff = out[c] - (double)target[3 * r + c];
      e += diff * diff;
    }
    photo[r] = e;
    dist[r] = out[5];
  });
  double sp = 0.0, sd = 0.0;
  for (int64_t r = 0; r < R; ++r) {
    sp += photo[r];
    sd += dist[r];
  }
  return sp / (3.0 * (double)R) + lambda * sd / (double)R;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): ten rounds of two 32x32 -> 64-bit products mixed into
// the 128-bit counter, the 64-bit key advanced by the Weyl constants between
// rounds.
void philox4x32_10(const uint32_t* ctr_in, const uint32_t* key_in, uint32_t* out) {
  const uint64_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  const uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += kW0;
      k[1] += kW1;
    }
    const uint64_t p0 = kM0 * c[0], p1 = kM1 * c[2];
    const uint32_t n0 = uint32_t(p1 >> 32) ^ c[1] ^ k[0];
    const uint32_t n1 = uint32_t(p1);
    const uint32_t n2 = uint32_t(p0 >> 32) ^ c[3] ^ k[1];
    const uint32_t n3 = uint32_t(p0);
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Point drawn in cell (cx, cy, cz) of region `region` at refresh `step`:
// counter (cell, region, step lo, step hi), key (seed lo, seed hi); each of the
// first three words gives xi = (word >> 8) / 2^24 in [0, 1) and
// u = ((float)c + xi) / G in FP32.
void cell_point(int64_t cell, int region, int32_t G, const int32_t* c3, int64_t step, uint64_t seed, float* u) {
  const uint32_t ctr[4] = {uint32_t(cell), uint32_t(region), uint32_t(uint64_t(step)),
                           uint32_t(uint64_t(step) >> 32)};
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  uint32_t r[4];
  philox4x32_10(ctr, key, r);
  for (int ax = 0; ax < 3; ++ax) {
    const float xi = (float)(r[ax] >> 8) * (1.0f / 16777216.0f);
    u[ax] = ((float)c3[ax] + xi) / (float)G;
  }
}

// ---------------------------------------------------------------------------
// Distance of a sample's hidden units from their ReLU kinks (a diagnostic for
// the gradient tests, not part of the method). A unit's pre-activation z is
// compared with the scale its rounding error grows with: the sum of the
// magnitudes of the products that form it, where each input carries its own
// scale forward (running error analysis: an input h computed from products of
// total magnitude s may be off by a multiple of s, not of |h|). For the fused
// MLP
//   s1_n = sum_i |feat_i W1_in|,   s2_m = sum_n |W2_nm| (h1_n + s1_n);
// for the split representation
//   s1_n = sum_i |feat_i Wd1_in|,  sg_m = sum_n |Wd2_nm| (h1_n + s1_n),
//   s2_n = sum_{m<16} |Wc1_mn| (|g_m| + sg_m) + sum_{m>=16} |Wc1_mn SH_m|,
//   s3_n = sum_i |Wc2_in| (h2_i + s2_i).
// The margin of a sample is min over units of |z| / s (a unit with s = 0 has
// z = 0 in any precision and counts as infinitely far).
double relu_margin_sample(const oracle_field& f, int region, const double* feat, const float* dir) {
  const int W = f.W, I = f.mlp_in;
  double best = INFINITY;
  auto take = [&](double z, double sc) {
    if (sc > 0.0) best = std::min(best, std::fabs(z) / sc);
  };
  if (f.arch == 1) {
    const double* Wd1 = f.mlp + int64_t(region) * density_params(I, W);
    const double* Wd2 = Wd1 + int64_t(I) * W;
    const double* Wc1 = f.mlp + int64_t(f.K) * density_params(I, W);
    const double* Wc2 = Wc1 + int64_t(kGeo + kSh) * W;
    std::vector<double> h1(W), s1(W), g(kGeo), sg(kGeo), h2(W), s2(W);
    for (int n = 0; n < W; ++n) {
      double z = 0.0, sc = 0.0;
      for (int i = 0; i < I; ++i) {
        z += feat[i] * Wd1[i * W + n];
        sc += std::fabs(feat[i] * Wd1[i * W + n]);
      }
      take(z, sc);
      h1[n] = z > 0.0 ? z : 0.0;
      s1[n] = sc;
    }
    for (int m = 0; m < kGeo; ++m) {
      double z = 0.0, sc = 0.0;
      for (int n = 0; n < W; ++n) {
        z += h1[n] * Wd2[n * kGeo + m];
        sc += std::fabs(Wd2[n * kGeo + m]) * (h1[n] + s1[n]);
      }
      g[m] = z;
      sg[m] = sc;
    }
    double sh[kSh];
    const double dd[3] = {(double)dir[0], (double)dir[1], (double)dir[2]};
    sh4(dd, sh);
    for (int n = 0; n < W; ++n) {
      double z = 0.0, sc = 0.0;
      for (int m = 0; m < kGeo; ++m) {
        z += g[m] * Wc1[m * W + n];
        sc += std::fabs(Wc1[m * W + n]) * (std::fabs(g[m]) + sg[m]);
      }
      for (int m = 0; m < kSh; ++m) {
        z += sh[m] * Wc1[(kGeo + m) * W + n];
        sc += std::fabs(sh[m] * Wc1[(kGeo + m) * W + n]);
      }
      take(z, sc);
      h2[n] = z > 0.0 ? z : 0.0;
      s2[n] = sc;
    }
    for (int n = 0; n < W; ++n) {
      double z = 0.0, sc = 0.0;
      for (int i = 0; i < W; ++i) {
        z += h2[i] * Wc2[i * W + n];
        sc += std::fabs(Wc2[i * W + n]) * (h2[i] + s2[i]);
      }
      take(z, sc);
    }
    return best;
  }
  const double* W1 = f.mlp + int64_t(region) * mlp_params(I, W);
  const double* W2 = W1 + int64_t(I) * W;
  std::vector<double> h1(W), s1(W);
  for (int n = 0; n < W; ++n) {
    double z = 0.0, sc = 0.0;
    for (int i = 0; i < I; ++i) {
      z += feat[i] * W1[i * W + n];
      sc += std::fabs(feat[i] * W1[i * W + n]);
    }
    take(z, sc);
    h1[n] = z > 0.0 ? z : 0.0;
    s1[n] = sc;
  }
  for (int m = 0; m < W; ++m) {
    double z = 0.0, sc = 0.0;
    for (int n = 0; n < W; ++n) {
      z += h1[n] * W2[n * W + m];
      sc += std::fabs(W2[n * W + m]) * (h1[n] + s1[n]);
    }
    take(z, sc);
  }
  return best;
}

}  // namespace

// ===========================================================================
extern "C" {

void oracle_set_threads(int n) { g_threads = n; }
int oracle_threads(void) { return n_threads(); }

int64_t oracle_table_entries(int32_t L, const int32_t* level_res, int32_t log2_T) {
  std::vector<Level> lv = make_levels(L, level_res, log2_T);
  return lv.back().offset + lv.back().size;
}
int64_t oracle_level_offset(int32_t L, const int32_t* level_res, int32_t log2_T, int32_t l) {
  return make_levels(L, level_res, log2_T)[l].offset;
}
int32_t oracle_level_dense(int32_t L, const int32_t* level_res, int32_t log2_T, int32_t l) {
  return make_levels(L, level_res, log2_T)[l].dense ? 1 : 0;
}
int64_t oracle_mlp_params(int32_t mlp_in, int32_t W) { return mlp_params(mlp_in, W); }
int64_t oracle_density_params(int32_t mlp_in, int32_t W) { return density_params(mlp_in, W); }
int64_t oracle_color_params(int32_t W) { return color_params(W); }

// Spherical harmonics of degrees 0..3 of n unit directions: out [n][16].
void oracle_sh4(int64_t n, const double* dirs, double* out) {
  for (int64_t i = 0; i < n; ++i) sh4(dirs + 3 * i, out + 16 * i);
}

// Segments of each ray, ray order. Outputs sized [R][K]; unused slots left as is.
void oracle_segments(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                     int32_t* nseg, int32_t* region, float* t0, float* t1, int32_t* nint) {
  parallel_for(R, [&](int64_t r, int) {
    std::vector<Seg> segs = ray_segments(*f, *s, ro + 3 * r, rd + 3 * r);
    std::vector<Interval> iv = ray_intervals(segs, s->S);
    nseg[r] = (int32_t)segs.size();
    for (size_t k = 0; k < segs.size(); ++k) {
      region[r * f->K + k] = segs[k].region;
      t0[r * f->K + k] = segs[k].t0;
      t1[r * f->K + k] = segs[k].t1;
      int32_t c = 0;
      for (auto& q : iv) c += (q.seg == (int)k);
      nint[r * f->K + k] = c;
    }
  });
}

// Intervals of each ray: count[R], a/b/region [R][max_int]. Returns -1 if any
// ray has more than max_int intervals.
int oracle_intervals(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                     int32_t max_int, int32_t* count, float* a, float* b, int32_t* region) {
  std::atomic<int> bad(0);
  parallel_for(R, [&](int64_t r, int) {
    std::vector<Interval> iv = ray_intervals(ray_segments(*f, *s, ro + 3 * r, rd + 3 * r), s->S);
    count[r] = (int32_t)iv.size();
    if ((int)iv.size() > max_int) {
      bad = 1;
      return;
    }
    for (size_t i = 0; i < iv.size(); ++i) {
      a[r * max_int + i] = iv[i].a;
      b[r * max_int + i] = iv[i].b;
      region[r * max_int + i] = iv[i].region;
    }
  });
  return bad ? -1 : 0;
}

// Per-sample level indices [R][max_int][L][8] (index within the level).
int oracle_hash_indices(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro,
                        const float* rd, int32_t max_int, uint32_t* idx) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  std::atomic<int> bad(0);
  parallel_for(R, [&](int64_t r, int) {
    const float* o = ro + 3 * r;
    const float* d = rd + 3 * r;
    std::vector<Interval> iv = ray_intervals(ray_segments(*f, *s, o, d), s->S);
    if ((int)iv.size() > max_int) {
      bad = 1;
      return;
    }
    Encoded enc;
    for (size_t i = 0; i < iv.size(); ++i) {
      const float tb = 0.5f * (iv[i].a + iv[i].b);
      float x[3];
      for (int ax = 0; ax < 3; ++ax) x[ax] = o[ax] + tb * d[ax];
      encode(*f, lv, iv[i].region, x, &enc);
      std::memcpy(idx + ((r * max_int + (int64_t)i) * f->L) * 8, enc.index.data(), sizeof(uint32_t) * f->L * 8);
    }
  });
  return bad ? -1 : 0;
}

// Encoding of explicit points: feat [n][mlp_in], idx [n][L][8] (may be NULL).
void oracle_encode_points(const oracle_field* f, int64_t n, const int32_t* region, const float* x, double* feat,
                          uint32_t* idx) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  parallel_for(n, [&](int64_t i, int) {
    Encoded enc;
    encode(*f, lv, region[i], x + 3 * i, &enc);
    std::memcpy(feat + i * f->mlp_in, enc.feat.data(), sizeof(double) * f->mlp_in);
    if (idx) std::memcpy(idx + i * f->L * 8, enc.index.data(), sizeof(uint32_t) * f->L * 8);
  });
}

// Raw MLP outputs o[n][4] for explicit features.
void oracle_mlp(const oracle_field* f, int64_t n, const int32_t* region, const double* feat, const float* dirs,
                double* o) {
  const float up[3] = {0.0f, 0.0f, 1.0f};
  parallel_for(n, [&](int64_t i, int) {
    MlpAct a;
    mlp_forward(*f, region[i], feat + i * f->mlp_in, dirs ? dirs + 3 * i : up, &a);
    for (int m = 0; m < 4; ++m) o[i * 4 + m] = a.o[m];
  });
}

// Render explicit interval values. seg_of[n] groups consecutive intervals into
// segments. out_single[7], out_part[7] as documented at render_single.
void oracle_render_samples(int64_t n, const int32_t* seg_of, const double* sigma, const double* rgb,
                           const double* tbar, const double* delta, double* out_single, double* out_part) {
  render_single((size_t)n, sigma, rgb, tbar, delta, out_single);
  render_partitioned((size_t)n, seg_of, sigma, rgb, tbar, delta, out_part);
}

// Segment-local partial {tau, C[3], A, D, L} of explicit interval values.
void oracle_render_local(int64_t n, const double* sigma, const double* rgb, const double* tbar, const double* delta,
                         double* part) {
  render_local((size_t)n, sigma, rgb, tbar, delta, part);
}

// Composite nseg partials [nseg][7] in order (Algorithm 1 and 2).
void oracle_composite(int64_t nseg, const double* parts, double* out) { composite((size_t)nseg, parts, out); }

// Full render of rays. mode 0: single pass (i); mode 1: partitioned (ii).
// rgb [R][3], depth/opacity/dist/tfinal [R]. n_samples [R] receives the
// number of samples evaluated on each ray: every interval, or with an
// occupancy grid those in occupied cells.
void oracle_render(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                   int32_t mode, double* rgb, double* depth, double* opacity, double* dist, double* tfinal,
                   int32_t* n_samples) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  parallel_for(R, [&](int64_t r, int) {
    RayEval re;
    eval_ray(*f, *s, lv, ro + 3 * r, rd + 3 * r, false, &re);
    double out[7];
    render_ray(re, mode, out);
    for (int c = 0; c < 3; ++c) rgb[3 * r + c] = out[c];
    depth[r] = out[3];
    opacity[r] = out[4];
    dist[r] = out[5];
    tfinal[r] = out[6];
    n_samples[r] = (int32_t)(re.iv.size() - std::count(re.skip.begin(), re.skip.end(), 1));
  });
}

// Loss = mean_{r,c} (C - C*)^2 + lambda * mean_r L_dist.
double oracle_loss(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                   const float* target, double lambda) {
  return loss_impl(*f, *s, R, ro, rd, target, lambda);
}

// Adjoint of the render for given output adjoints; g_tables [K][E][F] and
// g_mlp [K][P] are ACCUMULATED into.
void oracle_render_grad(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro,
                        const float* rd, const double* gC, const double* gD, const double* gA, const double* gL,
                        double* g_tables, double* g_mlp) {
  render_grad_impl(*f, *s, R, ro, rd, gC, gD, gA, gL, g_tables, g_mlp);
}

// Loss and its gradient (accumulated into g_tables / g_mlp). Returns the loss.
double oracle_loss_grad(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro,
                        const float* rd, const float* target, double lambda, double* g_tables, double* g_mlp) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  std::vector<double> gC(3 * R), gD(R, 0.0), gA(R, 0.0), gL(R, lambda / (double)R);
  std::vector<double> photo(R), dist(R);
  parallel_for(R, [&](int64_t r, int) {
    RayEval re;
    eval_ray(*f, *s, lv, ro + 3 * r, rd + 3 * r, false, &re);
    double out[7];
    render_ray(re, 0, out);
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double diff = out[c] - (double)target[3 * r + c];
      gC[3 * r + c] = 2.0 * diff / (3.0 * (double)R);
      e += diff * diff;
    }
    photo[r] = e;
    dist[r] = out[5];
  });
  render_grad_impl(*f, *s, R, ro, rd, gC.data(), gD.data(), gA.data(), gL.data(), g_tables, g_mlp);
  double sp = 0.0, sd = 0.0;
  for (int64_t r = 0; r < R; ++r) {
    sp += photo[r];
    sd += dist[r];
  }
  return sp / (3.0 * (double)R) + lambda * sd / (double)R;
}

// Central finite differences of the loss: for coordinate c, which[c] = 0
// selects tables[idx[c]], 1 selects mlp[idx[c]]. The field's arrays are
// perturbed in place (writable copies) and restored.
void oracle_fd_grad(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                    const float* target, double lambda, double* tables_rw, double* mlp_rw, int64_t n_coords,
                    const int32_t* which, const int64_t* idx, double eps, double* out) {
  oracle_field g = *f;
  g.tables = tables_rw;
  g.mlp = mlp_rw;
  for (int64_t c = 0; c < n_coords; ++c) {
    double* p = which[c] == 0 ? tables_rw + idx[c] : mlp_rw + idx[c];
    const double keep = *p;
    *p = keep + eps;
    const double lp = loss_impl(g, *s, R, ro, rd, target, lambda);
    *p = keep - eps;
    const double lm = loss_impl(g, *s, R, ro, rd, target, lambda);
    *p = keep;
    out[c] = (lp - lm) / (2.0 * eps);
  }
}

// Adam with bias correction, in place: m, v, p updated with gradient g at
// 1-based step t.
void oracle_adam(int64_t n, double* p, double* m, double* v, const double* g, int64_t t, double lr, double b1,
                 double b2, double eps) {
  const double c1 = 1.0 - std::pow(b1, (double)t);
  const double c2 = 1.0 - std::pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / c1;
    const double vh = v[i] / c2;
    p[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

// Analytic target field of isotropic Gaussian blobs, rendered single pass
// with the same intervals as the partitioned field:
//   sigma*(x) = sum_b a_b exp(-|x - mu_b|^2 / (2 s_b^2)),
//   c*(x) = sum_b a_b g_b(x) rgb_b / sigma*(x)   (0 where sigma* < 1e-12).
// blobs [nb][8] = mu xyz, s, a, rgb. Outputs rgb [R][3], depth [R], opacity [R].
void oracle_blob_render(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro,
                        const float* rd, int64_t nb, const double* blobs, double* rgb, double* depth,
                        double* opacity) {
  parallel_for(R, [&](int64_t r, int) {
    const float* o = ro + 3 * r;
    const float* d = rd + 3 * r;
    std::vector<Interval> iv = ray_intervals(ray_segments(*f, *s, o, d), s->S);
    double acc = 0.0, C[3] = {0, 0, 0}, A = 0, D = 0;
    for (size_t i = 0; i < iv.size(); ++i) {
      const float t = 0.5f * (iv[i].a + iv[i].b);
      const double dl = iv[i].b - iv[i].a;
      double x[3];
      for (int ax = 0; ax < 3; ++ax) x[ax] = (double)o[ax] + (double)t * (double)d[ax];
      double sig = 0.0, col[3] = {0, 0, 0};
      for (int64_t b = 0; b < nb; ++b) {
        const double* q = blobs + 8 * b;
        const double dx = x[0] - q[0], dy = x[1] - q[1], dz = x[2] - q[2];
        const double g = q[4] * std::exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * q[3] * q[3]));
        sig += g;
        for (int c = 0; c < 3; ++c) col[c] += g * q[5 + c];
      }
      const double tau = sig * dl;
      const double w = std::exp(-acc) * -std::expm1(-tau);
      for (int c = 0; c < 3; ++c) C[c] += w * (sig < 1e-12 ? 0.0 : col[c] / sig);
      A += w;
      D += w * (double)t;
      acc += tau;
    }
    for (int c = 0; c < 3; ++c) rgb[3 * r + c] = C[c];
    depth[r] = D;
    opacity[r] = A;
  });
}


// Philox4x32-10 of one counter / key (for known-answer checks).
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

// Occupancy-grid refresh of all K regions (grid G^3 per region, cells
// x-fastest: cell = x + G (y + G z)). density [K][G^3] is updated in place to
// max(decay * density, sigma(u_cell)); bits [K][ceil(G^3/32)] receive
// density > threshold (cell c in word c / 32, bit c % 32; unused bits 0).
// points (optional, [K][G^3][3]) receives the drawn region coordinates.
void oracle_occupancy_update(const oracle_field* f, int32_t G, int64_t step, uint64_t seed, double decay,
                             double threshold, double* density, uint32_t* bits, float* points) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  const int64_t cells = int64_t(G) * G * G;
  const int64_t words = (cells + 31) / 32;
  for (int64_t i = 0; i < int64_t(f->K) * words; ++i) bits[i] = 0u;
  std::vector<char> on(size_t(f->K) * cells, 0);
  parallel_for(int64_t(f->K) * cells, [&](int64_t i, int) {
    const int region = int(i / cells);
    const int64_t cell = i % cells;
    const int32_t c3[3] = {int32_t(cell % G), int32_t((cell / G) % G), int32_t(cell / (int64_t(G) * G))};
    float u[3];
    cell_point(cell, region, G, c3, step, seed, u);
    if (points)
      for (int ax = 0; ax < 3; ++ax) points[3 * i + ax] = u[ax];
    Encoded enc;
    MlpAct act;
    encode_u(*f, lv, region, u, &enc);
    const float up[3] = {0.0f, 0.0f, 1.0f};  // the density does not depend on the direction
    mlp_forward(*f, region, enc.feat.data(), up, &act);
    const double sigma = std::exp(act.o[0]);
    density[i] = std::max(decay * density[i], sigma);
    on[size_t(i)] = density[i] > threshold;
  });
  for (int64_t i = 0; i < int64_t(f->K) * cells; ++i)
    if (on[size_t(i)]) bits[(i / cells) * words + (i % cells) / 32] |= 1u << ((i % cells) % 32);
}


// Smallest ReLU margin (relu_margin_sample) over each ray's evaluated samples:
// margin [R], +inf for a ray without evaluated samples.
void oracle_relu_margin(const oracle_field* f, const oracle_sampling* s, int64_t R, const float* ro, const float* rd,
                        double* margin) {
  const std::vector<Level> lv = make_levels(f->L, f->level_res, f->log2_T);
  parallel_for(R, [&](int64_t r, int) {
    const float* o = ro + 3 * r;
    const float* d = rd + 3 * r;
    RayEval re;
    eval_ray(*f, *s, lv, o, d, true, &re);
    double best = INFINITY;
    for (size_t i = 0; i < re.iv.size(); ++i) {
      if (re.skip[i]) continue;
      best = std::min(best, relu_margin_sample(*f, re.iv[i].region, re.enc[i].feat.data(), d));
    }
    margin[r] = best;
  });
}

// Pinhole camera rays (the rays a render request asks for). cam = {origin[3],
// right[3], up[3], forward[3], tan_half_fov} as float32, the frame orthonormal;
// pixel p = i W + j (row i from the top, column j), p in [first, first +
// count). Prescribed FP32 operation sequence, one IEEE rounding per operation
// and no fused multiply-add (the GPU follows the same sequence, so the rays
// agree bit for bit):
//   aspect = W / H
//   x = ((((j + 0.5) / W) * 2 - 1) * tan) * aspect
//   y = (1 - ((i + 0.5) / H) * 2) * tan
//   v_a = (x right_a + y up_a) + forward_a
//   n = sqrt((v_0 v_0 + v_1 v_1) + v_2 v_2),   d_a = v_a / n,   o = origin.
void oracle_camera_rays(const float* cam, int32_t W, int32_t H, int64_t first, int64_t count, float* ro, float* rd) {
  const float* org = cam;
  const float* right = cam + 3;
  const float* up = cam + 6;
  const float* fwd = cam + 9;
  const float tan_h = cam[12];
  const float aspect = (float)W / (float)H;
  for (int64_t k = 0; k < count; ++k) {
    const int64_t p = first + k;
    const int32_t i = (int32_t)(p / W), j = (int32_t)(p % W);
    const float x = ((((float)j + 0.5f) / (float)W) * 2.0f - 1.0f) * tan_h * aspect;
    const float y = (1.0f - (((float)i + 0.5f) / (float)H) * 2.0f) * tan_h;
    float v[3];
    for (int a = 0; a < 3; ++a) v[a] = (x * right[a] + y * up[a]) + fwd[a];
    const float n = std::sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) {
      ro[3 * k + a] = org[a];
      rd[3 * k + a] = v[a] / n;
    }
  }
}

}  // extern "C"
