// Host-side check of the row-gather element walk (tests/test_walk_encoder_cpu.py).
//
// Reads a mesh (coordinates, positively oriented connectivity, velocities),
// builds every row's star independently (the positions of each incident
// element's other three nodes, listed as an even permutation), encodes it with
// the library's own encode_walk, and replays the walk the way the kernel runs
// it: a window of two nodes in registers (the newest node always enters q, p
// keeps its node or takes q's), orientation from the step byte, the carried
// cofactor with its sign, the next node's accumulator read BEFORE the leaving node's is
// written back (stale reads are simulated).  The replayed row sums (the
// convection + viscous entries w . c_x, the pressure-gradient sums of c_i and
// the determinant sum) must equal direct sums over the star in double.
//
// Usage: walk_replay <mesh file>; prints one summary line; exit code 0 when
// every row agrees to 1e-12 (row-scaled) and every element is evaluated once.
#include "../paper_2111_05651_gb300/csrc/nsi_create.cu"

#include <cstdio>

namespace nsi {
int gather_kernel_regs(int) { return 64; }  // the launch planner is not exercised here
}  // namespace nsi

namespace {

struct P3 {
  double x, y, z;
};
P3 sub3(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
P3 cross3(P3 a, P3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double dot3(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

}  // namespace

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* fp = std::fopen(argv[1], "rb");
  if (!fp) return 2;
  int64_t n = 0, E = 0;
  if (std::fread(&n, 8, 1, fp) != 1 || std::fread(&E, 8, 1, fp) != 1) return 2;
  std::vector<P3> X(n), Uv(n);
  std::vector<int32_t> ln(4 * E);
  if (std::fread(X.data(), 24, n, fp) != (size_t)n || std::fread(ln.data(), 4, 4 * E, fp) != (size_t)(4 * E) ||
      std::fread(Uv.data(), 24, n, fp) != (size_t)n)
    return 2;
  std::fclose(fp);

  std::vector<std::vector<std::pair<int64_t, int>>> inc(n);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 4; ++a) inc[ln[4 * e + a]].push_back({e, a});
  static const int EVEN[4][3] = {{1, 2, 3}, {0, 3, 2}, {3, 0, 1}, {2, 1, 0}};
  const double kc = 1.0 / 120.0, kmu = 1e-3 / 6.0;

  nsi::WalkWork ws;
  int64_t steps = 0, elems = 0, paths_rows = 0, skipped = 0, stale = 0;
  double worst = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int32_t> col;
    for (auto& ea : inc[i])
      for (int a = 0; a < 4; ++a) col.push_back(ln[4 * ea.first + a]);
    std::sort(col.begin(), col.end());
    col.erase(std::unique(col.begin(), col.end()), col.end());
    const int len = (int)col.size();
    if (len == 0) continue;
    if (len > nsi::STAR_MAX_ROW) {
      ++skipped;
      continue;
    }
    auto pos = [&](int32_t j) { return (int)(std::lower_bound(col.begin(), col.end(), j) - col.begin()); };
    const int dp = pos((int32_t)i);
    std::vector<uint16_t> tri;
    for (auto& ea : inc[i]) {
      unsigned w = 0;
      for (int m2 = 0; m2 < 3; ++m2) w |= unsigned(pos(ln[4 * ea.first + EVEN[ea.second][m2]])) << (5 * m2);
      tri.push_back((uint16_t)w);
    }
    std::vector<uint8_t> out;
    if (!nsi::encode_walk(tri.data(), (int)tri.size(), dp, out, ws)) {
      std::printf("FAIL encode row %lld\n", (long long)i);
      return 1;
    }
    steps += (int64_t)out.size();
    elems += (int64_t)tri.size();
    int nel = 0, fills = 0;
    for (uint8_t b : out) {
      nel += (b & nsi::WALK_ELEM) != 0;
      fills += (b & nsi::WALK_ELEM) == 0;
    }
    if (nel != (int)tri.size()) {
      std::printf("FAIL row %lld: %d elements walked, %zu in the star\n", (long long)i, nel, tri.size());
      return 1;
    }
    paths_rows += fills > 2;
    // direct sums over the star
    const P3 u2i{2 * Uv[i].x, 2 * Uv[i].y, 2 * Uv[i].z};
    std::vector<double> A(len, 0), Gx(len, 0), Gy(len, 0), Gz(len, 0);
    double D = 0;
    for (uint16_t w : tri) {
      const int ps[3] = {w & 31, (w >> 5) & 31, (w >> 10) & 31};
      P3 d[3], c[3];
      for (int b = 0; b < 3; ++b) d[b] = sub3(X[col[ps[b]]], X[i]);
      c[0] = cross3(d[1], d[2]);
      c[1] = cross3(d[2], d[0]);
      c[2] = cross3(d[0], d[1]);
      const double det = dot3(d[0], c[0]);
      const P3 ci{-(c[0].x + c[1].x + c[2].x), -(c[0].y + c[1].y + c[2].y), -(c[0].z + c[1].z + c[2].z)};
      const double kv = kmu / det;
      P3 us = u2i;
      for (int b = 0; b < 3; ++b) us = {us.x + Uv[col[ps[b]]].x, us.y + Uv[col[ps[b]]].y, us.z + Uv[col[ps[b]]].z};
      const P3 w3{kc * us.x + kv * ci.x, kc * us.y + kv * ci.y, kc * us.z + kv * ci.z};
      for (int b = 0; b < 3; ++b) {
        A[ps[b]] += dot3(w3, c[b]);
        Gx[ps[b]] += ci.x;
        Gy[ps[b]] += ci.y;
        Gz[ps[b]] += ci.z;
      }
      D += det;
    }
    // the kernel's walk: shared-memory slots, window registers, prefetch
    struct Node {
      int k;
      P3 d, u;
      double a, gx, gy, gz;
    };
    std::vector<double> sA(len, 0), sX(len, 0), sY(len, 0), sZ(len, 0);
    std::vector<int> held(len, 0);  // nodes currently in registers (a read of one would be stale)
    double sD = 0;
    auto load = [&](int k) {
      if (k != dp && held[k]) ++stale;
      ++held[k];
      return Node{k, sub3(X[col[k]], X[i]), Uv[col[k]], sA[k], sX[k], sY[k], sZ[k]};
    };
    auto store = [&](const Node& nd) {
      --held[nd.k];
      sA[nd.k] = nd.a;
      sX[nd.k] = nd.gx;
      sY[nd.k] = nd.gy;
      sZ[nd.k] = nd.gz;
    };
    // the first two steps only fill the window: the kernel loads their nodes
    // directly, with the first element's carried cofactor d_p x d_q
    if (out.size() < 3 || (out[0] & nsi::WALK_ELEM) || (out[1] & nsi::WALK_ELEM)) {
      std::printf("FAIL row %lld: the walk does not start with two filling steps\n", (long long)i);
      return 1;
    }
    Node p = load(out[0] & nsi::WALK_POS), q = load(out[1] & nsi::WALK_POS);
    P3 m = cross3(p.d, q.d);
    double sg = -1.0;  // c_c = -sg m
    unsigned w = out[2];
    Node c = load(w & nsi::WALK_POS);
    const size_t ns = out.size();
    for (size_t s = 2; s < ns; ++s) {
      const bool last = s + 1 >= ns;
      const unsigned wn = last ? w : out[s + 1];
      Node cn{};
      if (!last) cn = load(wn & nsi::WALK_POS);  // before this step's write-back
      const P3 cp = cross3(q.d, c.d), cq = cross3(c.d, p.d);
      if (w & nsi::WALK_ELEM) {
        const double det = dot3(p.d, cp);
        const P3 ci{sg * m.x - cp.x - cq.x, sg * m.y - cp.y - cq.y, sg * m.z - cp.z - cq.z};
        const double kv = kmu / det;
        const P3 w3{kc * (u2i.x + p.u.x + q.u.x + c.u.x) + kv * ci.x, kc * (u2i.y + p.u.y + q.u.y + c.u.y) + kv * ci.y,
                    kc * (u2i.z + p.u.z + q.u.z + c.u.z) + kv * ci.z};
        const double f = (w & nsi::WALK_NEG) ? -1.0 : 1.0;
        p.a += f * dot3(w3, cp);
        q.a += f * dot3(w3, cq);
        c.a += -f * sg * dot3(w3, m);
        for (Node* nd : {&p, &q, &c}) {
          nd->gx += f * ci.x;
          nd->gy += f * ci.y;
          nd->gz += f * ci.z;
        }
        sD += f * det;
      }
      if (w & nsi::WALK_EVQ) {  // q leaves
        store(q);
        m = cq;
        sg = 1.0;
      } else {  // p leaves, q's node moves to p
        store(p);
        p = q;
        m = cp;
        sg = -1.0;
      }
      q = c;  // the newest node is always q
      if (!last) c = cn;
      w = wn;
    }
    store(p);
    store(q);
    double sc = 0, gs = 0;  // row scales of A and of the pressure-gradient sums
    for (int k = 0; k < len; ++k) {
      sc = std::max(sc, std::fabs(A[k]));
      gs = std::max(gs, std::max(std::fabs(Gx[k]), std::max(std::fabs(Gy[k]), std::fabs(Gz[k]))));
    }
    for (int k = 0; k < len; ++k) {
      if (k == dp) {
        if (sA[k] != 0 || sX[k] != 0 || sY[k] != 0 || sZ[k] != 0) {
          std::printf("FAIL row %lld: diagonal slot written\n", (long long)i);
          return 1;
        }
        continue;
      }
      worst = std::max(worst, std::fabs(sA[k] - A[k]) / sc);
      const double ge = std::max(std::fabs(sX[k] - Gx[k]), std::max(std::fabs(sY[k] - Gy[k]), std::fabs(sZ[k] - Gz[k])));
      worst = std::max(worst, ge / gs);
    }
    worst = std::max(worst, std::fabs(sD - D) / std::fabs(D));
  }
  std::printf("rows=%lld elements=%lld steps=%lld steps_per_element=%.4f multipath_rows=%lld skipped=%lld "
              "stale_reads=%lld worst=%.3g\n",
              (long long)n, (long long)elems, (long long)steps, elems ? (double)steps / elems : 0.0,
              (long long)paths_rows, (long long)skipped, (long long)stale, worst);
  return (worst <= 1e-12 && stale == 0) ? 0 : 1;
}
