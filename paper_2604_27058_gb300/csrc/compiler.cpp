// compiler.cpp — offline Clifford-frame compiler (host C++).
//
// Turns extended-Stim text into the SVM bytecode of program.h (Sec. 3.1):
//   1. parse + unroll REPEAT, assigning physical event / record / noise-site
//      indices (the keys of the random draws);
//   2. Heisenberg-map every active operation through the Clifford frame
//      (Def. 1): the frame is kept as the images M(X_j), M(Z_j) of the
//      physical generators under P -> U_C^dagger P U_C;
//   3. Pauli-localise mapped generators (Lemma 1, App. A; dormant pivot
//      preferred, Lemma 2) and absorb V into the frame (U_C <- U_C V^dagger);
//   4. emit bytecode (frame ops, expansion fused with the rotation as in
//      OP_EXPAND_T, array ops, dormant/active measurements, coalesced noise
//      blocks, records), noise survival tables and record-slot assignment.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "compiler.h"

namespace nc {

// ---------------------------------------------------------------------------
// Parser
// ---------------------------------------------------------------------------
namespace {

struct CompileError : std::runtime_error {
  int code;
  CompileError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

[[noreturn]] void fail(int code, const std::string& msg) { throw CompileError(code, msg); }

enum Kind { K_GATE, K_ROT, K_MEAS, K_NOISE, K_FF, K_DET, K_OBS, K_PROBE };

struct PhysOp {
  Kind kind = K_GATE;
  std::string name;   // canonical gate / channel name
  int q0 = -1, q1 = -1;
  double arg = 0.0;   // rotation angle or probability
  int64_t event = -1, record = -1, site = -1;
  bool reset = false;
  bool xbasis = false;
  std::vector<int64_t> recs;  // det / obs records; ff: recs[0]; probe: its qubits
  int64_t index = -1;         // detector / observable / probe index
  int instr = -1;     // source instruction ordinal (groups targets of one line)
};

struct Line {
  std::string name;
  std::vector<double> args;
  std::vector<std::string> targets;
  int repeat = -1;              // >= 0: REPEAT block
  std::vector<Line> body;
};

std::string upper(std::string s) {
  for (auto& c : s) c = (char)toupper((unsigned char)c);
  return s;
}

std::string trim(const std::string& s) {
  size_t a = s.find_first_not_of(" \t\r");
  if (a == std::string::npos) return "";
  size_t b = s.find_last_not_of(" \t\r");
  return s.substr(a, b - a + 1);
}

std::vector<std::string> split_ws(const std::string& s) {
  std::vector<std::string> out;
  size_t i = 0;
  while (i < s.size()) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t')) i++;
    size_t j = i;
    while (j < s.size() && s[j] != ' ' && s[j] != '\t') j++;
    if (j > i) out.push_back(s.substr(i, j - i));
    i = j;
  }
  return out;
}

double parse_double(const std::string& t) {
  const char* s = t.c_str();
  char* end = nullptr;
  double v = strtod(s, &end);
  if (end == s || *end != 0 || !std::isfinite(v)) fail(1, "bad number '" + t + "'");
  return v;
}

std::vector<Line> parse_lines(const std::vector<std::string>& lines, size_t& pos, int depth) {
  std::vector<Line> out;
  while (pos < lines.size()) {
    std::string line = lines[pos];
    if (line == "}") {
      if (depth == 0) fail(1, "unmatched '}'");
      pos++;
      return out;
    }
    std::string up = upper(line);
    if (up.rfind("REPEAT", 0) == 0 && (up.size() == 6 || up[6] == ' ' || up[6] == '\t')) {
      auto toks = split_ws(line);
      if (toks.size() != 3 || toks[2] != "{") fail(1, "bad REPEAT line: " + line);
      char* end = nullptr;
      long n = strtol(toks[1].c_str(), &end, 10);
      if (*end != 0 || n < 0) fail(1, "bad REPEAT count: " + line);
      pos++;
      Line blk;
      blk.repeat = (int)n;
      blk.body = parse_lines(lines, pos, depth + 1);
      out.push_back(std::move(blk));
      continue;
    }
    Line l;
    size_t i = 0;
    while (i < line.size() && (isalnum((unsigned char)line[i]) || line[i] == '_')) i++;
    if (i == 0) fail(1, "cannot parse line: " + line);
    l.name = upper(line.substr(0, i));
    std::string rest = line.substr(i);
    if (!rest.empty() && rest[0] == '(') {
      size_t close = rest.find(')');
      if (close == std::string::npos) fail(1, "missing ')': " + line);
      std::string inner = rest.substr(1, close - 1);
      size_t s = 0;
      while (s <= inner.size()) {
        size_t c = inner.find(',', s);
        std::string tok = trim(inner.substr(s, c == std::string::npos ? std::string::npos : c - s));
        if (!tok.empty()) l.args.push_back(parse_double(tok));
        if (c == std::string::npos) break;
        s = c + 1;
      }
      rest = rest.substr(close + 1);
    }
    l.targets = split_ws(rest);
    out.push_back(std::move(l));
    pos++;
  }
  if (depth) fail(1, "unterminated REPEAT block");
  return out;
}

const std::map<std::string, std::string>& aliases() {
  static const std::map<std::string, std::string> a = {
      {"CNOT", "CX"}, {"ZCX", "CX"}, {"ZCY", "CY"}, {"ZCZ", "CZ"}, {"MZ", "M"},
      {"RZ", "R"}, {"MRZ", "MR"}, {"SQRT_Z", "S"}, {"SQRT_Z_DAG", "S_DAG"}};
  return a;
}

bool is_1q_clifford(const std::string& n) {
  static const char* v[] = {"I", "H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG",
                            "SQRT_Y", "SQRT_Y_DAG"};
  for (auto s : v)
    if (n == s) return true;
  return false;
}
bool is_2q_clifford(const std::string& n) {
  return n == "CX" || n == "CY" || n == "CZ" || n == "SWAP";
}

struct Flattener {
  std::vector<PhysOp> ops;
  int64_t n_q = 0, ev = 0, rec = 0, site = 0, det = 0, n_obs = 0, probe = 0;
  int instr = 0;
  std::vector<double> site_p;
  std::vector<uint8_t> site_kind;

  int64_t rec_target(const std::string& t) {
    if (t.rfind("rec[-", 0) != 0 || t.back() != ']') fail(1, "bad record target '" + t + "'");
    std::string num = t.substr(5, t.size() - 6);
    char* end = nullptr;
    long k = strtol(num.c_str(), &end, 10);
    if (*end != 0 || k < 1 || k > rec) fail(1, "record target out of range '" + t + "'");
    return rec - k;
  }
  int qubit(const std::string& t) {
    if (t.empty()) fail(1, "empty target");
    for (char c : t)
      if (!isdigit((unsigned char)c)) fail(1, "bad qubit target '" + t + "'");
    long q = strtol(t.c_str(), nullptr, 10);
    if (q >= (long)kMaxQubits) fail(2, "qubit index above the supported maximum");
    n_q = std::max<int64_t>(n_q, q + 1);
    return (int)q;
  }

  void run(const std::vector<Line>& block) {
    for (auto& l : block) {
      if (l.repeat >= 0) {
        for (int r = 0; r < l.repeat; r++) run(l.body);
        continue;
      }
      one(l);
      instr++;
    }
  }

  void one(const Line& l) {
    std::string name = l.name;
    auto al = aliases().find(name);
    if (al != aliases().end()) name = al->second;
    if (name == "TICK" || name == "QUBIT_COORDS" || name == "SHIFT_COORDS") return;
    if (name == "DETECTOR") {
      PhysOp o; o.kind = K_DET;
      for (auto& t : l.targets) o.recs.push_back(rec_target(t));
      o.index = det++;
      ops.push_back(o);
      return;
    }
    if (name == "EXPVAL") {
      // one probe per Pauli-product target, e.g. X0*Y1*Z5 (letters in name)
      if (!l.args.empty() || l.targets.empty()) fail(1, "EXPVAL takes Pauli product targets and no argument");
      for (auto& t : l.targets) {
        PhysOp o; o.kind = K_PROBE;
        size_t s0 = 0;
        while (s0 <= t.size()) {
          size_t c = t.find('*', s0);
          std::string f = t.substr(s0, c == std::string::npos ? std::string::npos : c - s0);
          if (f.size() < 2 || (f[0] != 'X' && f[0] != 'Y' && f[0] != 'Z')) fail(1, "bad Pauli product target '" + t + "'");
          int q = qubit(f.substr(1));
          for (auto r : o.recs)
            if (r == q) fail(1, "qubit repeated in '" + t + "'");
          o.recs.push_back(q);
          o.name.push_back(f[0]);
          if (c == std::string::npos) break;
          s0 = c + 1;
        }
        o.index = probe++;
        o.instr = instr;
        ops.push_back(o);
      }
      return;
    }
    if (name == "OBSERVABLE_INCLUDE") {
      if (l.args.size() != 1 || l.args[0] < 0 || l.args[0] != std::floor(l.args[0]))
        fail(1, "OBSERVABLE_INCLUDE needs one integer index");
      PhysOp o; o.kind = K_OBS;
      o.index = (int64_t)l.args[0];
      if (o.index > 1 << 20) fail(2, "observable index too large");
      for (auto& t : l.targets) o.recs.push_back(rec_target(t));
      n_obs = std::max(n_obs, o.index + 1);
      ops.push_back(o);
      return;
    }
    bool has_rec = false;
    for (auto& t : l.targets)
      if (t.rfind("rec[", 0) == 0) has_rec = true;
    if ((name == "CX" || name == "CY" || name == "CZ") && has_rec) {
      if (l.targets.size() % 2) fail(1, name + " needs target pairs");
      for (size_t k = 0; k < l.targets.size(); k += 2) {
        const auto &a = l.targets[k], &b = l.targets[k + 1];
        PhysOp o; o.kind = K_FF;
        o.name = name == "CX" ? "X" : name == "CY" ? "Y" : "Z";
        o.instr = instr;
        if (a.rfind("rec[", 0) == 0 && b.rfind("rec[", 0) != 0) {
          o.recs.push_back(rec_target(a));
          o.q0 = qubit(b);
        } else if (name == "CZ" && b.rfind("rec[", 0) == 0 && a.rfind("rec[", 0) != 0) {
          o.recs.push_back(rec_target(b));
          o.q0 = qubit(a);
        } else {
          fail(2, "unsupported classical control in " + name);
        }
        ops.push_back(o);
      }
      return;
    }
    std::vector<int> qs;
    for (auto& t : l.targets) qs.push_back(qubit(t));
    if (is_1q_clifford(name)) {
      if (!l.args.empty()) fail(1, name + " takes no argument");
      for (int q : qs) {
        PhysOp o; o.kind = K_GATE;
        o.name = name;
        o.q0 = q;
        o.instr = instr;
        ops.push_back(o);
      }
    } else if (is_2q_clifford(name)) {
      if (qs.size() % 2) fail(1, name + " needs target pairs");
      for (size_t k = 0; k < qs.size(); k += 2) {
        if (qs[k] == qs[k + 1]) fail(1, name + " on the same qubit twice");
        PhysOp o; o.kind = K_GATE;
        o.name = name;
        o.q0 = qs[k];
        o.q1 = qs[k + 1];
        o.instr = instr;
        ops.push_back(o);
      }
    } else if (name == "T" || name == "T_DAG" || name == "R_Z" || name == "R_X" || name == "R_Y") {
      bool t = name == "T" || name == "T_DAG";
      if (t && !l.args.empty()) fail(1, name + " takes no argument");
      if (!t && l.args.size() != 1) fail(1, name + " needs one angle");
      for (int q : qs) {
        PhysOp o; o.kind = K_ROT;
        o.name = name;
        o.q0 = q;
        o.arg = t ? 0.0 : l.args[0];
        o.instr = instr;
        ops.push_back(o);
      }
    } else if (name == "M" || name == "MX" || name == "MR" || name == "R") {
      double p = 0.0;
      if (!l.args.empty()) {
        if (name == "R" || l.args.size() != 1) fail(1, "bad arguments for " + name);
        p = l.args[0];
        if (!(p >= 0.0 && p <= 1.0)) fail(1, "probability out of range");
      }
      for (int q : qs) {
        PhysOp o; o.kind = K_MEAS;
        o.name = name;
        o.q0 = q;
        o.xbasis = name == "MX";
        o.reset = name == "R" || name == "MR";
        o.event = ev++;
        o.instr = instr;
        if (name != "R") {
          o.record = rec++;
          if (p > 0) {
            o.site = site++;
            o.arg = p;
            site_p.push_back(p);
            site_kind.push_back(SITE_FLIP);
          }
        }
        ops.push_back(o);
      }
    } else if (name == "X_ERROR" || name == "Y_ERROR" || name == "Z_ERROR" ||
               name == "DEPOLARIZE1" || name == "DEPOLARIZE2") {
      if (l.args.size() != 1 || !(l.args[0] >= 0.0 && l.args[0] <= 1.0))
        fail(1, "bad probability for " + name);
      int width = name == "DEPOLARIZE2" ? 2 : 1;
      if (qs.size() % width) fail(1, name + " needs target pairs");
      uint8_t kind = name == "X_ERROR" ? SITE_X : name == "Y_ERROR" ? SITE_Y
                   : name == "Z_ERROR" ? SITE_Z : name == "DEPOLARIZE1" ? SITE_D1 : SITE_D2;
      for (size_t k = 0; k < qs.size(); k += width) {
        PhysOp o; o.kind = K_NOISE;
        o.name = name;
        o.q0 = qs[k];
        o.q1 = width == 2 ? qs[k + 1] : -1;
        o.arg = l.args[0];
        o.site = site++;
        o.instr = instr;
        site_p.push_back(l.args[0]);
        site_kind.push_back(kind);
        ops.push_back(o);
      }
    } else {
      fail(2, "unsupported instruction " + name);
    }
  }
};

// ---------------------------------------------------------------------------
// Pauli algebra: i^ph X^x Z^z, X^x Z^z = prod_j X_j^x_j prod_j Z_j^z_j
// ---------------------------------------------------------------------------
struct Pauli {
  std::vector<uint64_t> x, z;
  int ph = 0;
  explicit Pauli(int nw = 0) : x(nw, 0), z(nw, 0) {}
  bool xb(int q) const { return (x[q >> 6] >> (q & 63)) & 1; }
  bool zb(int q) const { return (z[q >> 6] >> (q & 63)) & 1; }
  void setx(int q, bool v) {
    uint64_t m = 1ull << (q & 63);
    x[q >> 6] = v ? (x[q >> 6] | m) : (x[q >> 6] & ~m);
  }
  void setz(int q, bool v) {
    uint64_t m = 1ull << (q & 63);
    z[q >> 6] = v ? (z[q >> 6] | m) : (z[q >> 6] & ~m);
  }
  bool xzero() const {
    for (auto w : x)
      if (w) return false;
    return true;
  }
};

int popc64(uint64_t v) { return __builtin_popcountll(v); }

// a <- a * b
void pmul_inplace(Pauli& a, const Pauli& b) {
  int c = 0;
  for (size_t w = 0; w < a.x.size(); w++) c += popc64(a.z[w] & b.x[w]);
  a.ph = (a.ph + b.ph + 2 * c) & 3;
  for (size_t w = 0; w < a.x.size(); w++) {
    a.x[w] ^= b.x[w];
    a.z[w] ^= b.z[w];
  }
}

// Hermitian sign bit of (-1)^s prod sigma_j written as i^ph X^x Z^z.
int herm_sign(const Pauli& p) {
  int xz = 0;
  for (size_t w = 0; w < p.x.size(); w++) xz += popc64(p.x[w] & p.z[w]);
  int d = ((p.ph - xz) % 4 + 4) % 4;
  if (d != 0 && d != 2) fail(9, "non-Hermitian Pauli in the compiler");
  return d / 2;
}

// ---------------------------------------------------------------------------
// Gate conjugation tables, derived numerically from the gate unitaries.
// Local qubit 0 is the more significant bit of the 4x4 basis index.
// ---------------------------------------------------------------------------
using cd = std::complex<double>;
struct Mat {
  int n;
  cd a[16];
};

Mat mat1(const std::string& g) {
  Mat m{2, {}};
  const double s = 1.0 / std::sqrt(2.0);
  auto set = [&](cd a, cd b, cd c, cd d) { m.a[0] = a; m.a[1] = b; m.a[2] = c; m.a[3] = d; };
  const cd I(0, 1);
  if (g == "I") set(1, 0, 0, 1);
  else if (g == "H") set(s, s, s, -s);
  else if (g == "S") set(1, 0, 0, I);
  else if (g == "S_DAG") set(1, 0, 0, -I);
  else if (g == "X") set(0, 1, 1, 0);
  else if (g == "Y") set(0, -I, I, 0);
  else if (g == "Z") set(1, 0, 0, -1);
  else if (g == "SQRT_X") set(0.5 * (1.0 + I), 0.5 * (1.0 - I), 0.5 * (1.0 - I), 0.5 * (1.0 + I));
  else if (g == "SQRT_X_DAG") set(0.5 * (1.0 - I), 0.5 * (1.0 + I), 0.5 * (1.0 + I), 0.5 * (1.0 - I));
  else if (g == "SQRT_Y") set(0.5 * (1.0 + I), -0.5 * (1.0 + I), 0.5 * (1.0 + I), 0.5 * (1.0 + I));
  else if (g == "SQRT_Y_DAG") set(0.5 * (1.0 - I), 0.5 * (1.0 - I), -0.5 * (1.0 - I), 0.5 * (1.0 - I));
  else fail(9, "no matrix for " + g);
  return m;
}

Mat mat2(const std::string& g) {
  Mat m{4, {}};
  const cd I(0, 1);
  for (int ia = 0; ia < 2; ia++)
    for (int ib = 0; ib < 2; ib++) {
      int src = 2 * ia + ib;
      if (g == "CX") m.a[(2 * ia + (ib ^ ia)) * 4 + src] = 1;
      else if (g == "CZ") m.a[src * 4 + src] = (ia && ib) ? -1 : 1;
      else if (g == "SWAP") m.a[(2 * ib + ia) * 4 + src] = 1;
      else if (g == "CY") {
        if (!ia) m.a[src * 4 + src] = 1;
        else m.a[(2 + (1 - ib)) * 4 + src] = ib == 0 ? I : -I;
      } else fail(9, "no matrix for " + g);
    }
  return m;
}

Mat mmul(const Mat& a, const Mat& b) {
  Mat c{a.n, {}};
  for (int i = 0; i < a.n; i++)
    for (int j = 0; j < a.n; j++) {
      cd s = 0;
      for (int k = 0; k < a.n; k++) s += a.a[i * a.n + k] * b.a[k * a.n + j];
      c.a[i * a.n + j] = s;
    }
  return c;
}
Mat dag(const Mat& a) {
  Mat c{a.n, {}};
  for (int i = 0; i < a.n; i++)
    for (int j = 0; j < a.n; j++) c.a[i * a.n + j] = std::conj(a.a[j * a.n + i]);
  return c;
}

// Local Pauli matrix X^x Z^z over w qubits (local qubit 0 most significant).
Mat local_pauli(int lx, int lz, int w) {
  Mat single[4];
  single[0] = mat1("I");
  single[1] = mat1("X");
  single[2] = mat1("Z");
  single[3] = mmul(mat1("X"), mat1("Z"));
  // factor j (j = 0 most significant) reads bit (w - 1 - j) of lx / lz
  auto idx = [&](int j) {
    int bit = w - 1 - j;
    return ((lx >> bit) & 1) | (((lz >> bit) & 1) << 1);
  };
  Mat out = single[idx(0)];
  if (w == 2) {
    Mat b = single[idx(1)];
    Mat k{4, {}};
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++)
        for (int r = 0; r < 2; r++)
          for (int c = 0; c < 2; c++) k.a[(2 * i + r) * 4 + (2 * j + c)] = out.a[i * 2 + j] * b.a[r * 2 + c];
    out = k;
  }
  return out;
}

struct LocalPauli {
  int x, z, ph;
};

LocalPauli identify(const Mat& m, int w) {
  for (int lx = 0; lx < (1 << w); lx++)
    for (int lz = 0; lz < (1 << w); lz++) {
      Mat b = local_pauli(lx, lz, w);
      for (int ph = 0; ph < 4; ph++) {
        cd f = ph == 0 ? cd(1, 0) : ph == 1 ? cd(0, 1) : ph == 2 ? cd(-1, 0) : cd(0, -1);
        bool ok = true;
        for (int i = 0; i < m.n * m.n && ok; i++)
          if (std::abs(m.a[i] - f * b.a[i]) > 1e-9) ok = false;
        if (ok) return {lx, lz, ph};
      }
    }
  fail(9, "conjugation did not give a Pauli");
}

// Table for G^dagger g G (inverse=true) or G g G^dagger, g = X_0, Z_0, X_1, Z_1.
struct ConjTable {
  int w;
  LocalPauli img[4];
};

const ConjTable& conj_table(const std::string& g, bool inverse) {
  static std::map<std::pair<std::string, bool>, ConjTable> cache;
  auto key = std::make_pair(g, inverse);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  Mat u = is_2q_clifford(g) ? mat2(g) : mat1(g);
  int w = u.n == 4 ? 2 : 1;
  if (inverse) u = dag(u);
  ConjTable t{w, {}};
  for (int j = 0; j < w; j++)
    for (int k = 0; k < 2; k++) {
      // local qubit j is bit (w-1-j) of the local Pauli index (qubit 0 most significant)
      int bit = 1 << (w - 1 - j);
      Mat gm = local_pauli(k == 0 ? bit : 0, k == 1 ? bit : 0, w);
      t.img[2 * j + k] = identify(mmul(mmul(u, gm), dag(u)), w);
    }
  return cache[key] = t;
}

// ---------------------------------------------------------------------------
// Compiler state
// ---------------------------------------------------------------------------
struct Emitted {
  Op op;
  std::vector<int64_t> uses;  // record ids read by this op
  int64_t def = -1;           // record id written by this op
};

struct Compiler {
  int n = 0, nw64 = 0, nw32 = 0;
  std::vector<Pauli> img;  // img[2j] = M(X_j), img[2j+1] = M(Z_j)
  std::vector<int> act;    // position -> virtual qubit
  std::vector<int> pos_of; // virtual qubit -> position or -1
  std::vector<Emitted> code;
  std::vector<uint32_t> masks;  // 32-bit words
  uint32_t k_max = 0;
  // noise
  std::vector<double> site_p;
  std::vector<uint8_t> site_kind;
  std::vector<uint32_t> site_eff;   // mask offset of option 0, or flip record id
  std::vector<int64_t> site_flip_id;
  // records
  int64_t next_id = 0;
  std::vector<int64_t> record_id;   // physical record -> id
  std::vector<int64_t> pending_out; // ids awaiting REC_OUT (after their flip block)
  std::vector<int64_t> pending_row;
  nc_info_counts counts{};

  explicit Compiler(int nq) : n(std::max(1, nq)) {
    nw64 = (n + 63) / 64;
    nw32 = (n + 31) / 32;
    img.assign(2 * n, Pauli(nw64));
    for (int j = 0; j < n; j++) {
      img[2 * j].setx(j, true);
      img[2 * j + 1].setz(j, true);
    }
    pos_of.assign(n, -1);
  }

  // M(P) for P = i^ph X^lx Z^lz on physical qubits qs (local bit j <-> qs[j],
  // local qubit 0 most significant as in the conjugation tables).
  Pauli map_local(const std::vector<int>& qs, int lx, int lz, int ph) {
    int w = (int)qs.size();
    Pauli acc(nw64);
    acc.ph = ph & 3;
    for (int j = 0; j < w; j++)
      if ((lx >> (w - 1 - j)) & 1) pmul_inplace(acc, img[2 * qs[j]]);
    for (int j = 0; j < w; j++)
      if ((lz >> (w - 1 - j)) & 1) pmul_inplace(acc, img[2 * qs[j] + 1]);
    return acc;
  }

  // M(P) for a Pauli P = i^ph X^x Z^z given by its bits (the images of its
  // X factors, then of its Z factors, in that order).
  Pauli map_pauli(const Pauli& q) const {
    Pauli acc(nw64);
    acc.ph = q.ph & 3;
    for (int j = 0; j < n; j++)
      if (q.xb(j)) pmul_inplace(acc, img[2 * j]);
    for (int j = 0; j < n; j++)
      if (q.zb(j)) pmul_inplace(acc, img[2 * j + 1]);
    return acc;
  }

  Pauli map_letter(int q, char l) {
    // X = X, Z = Z, Y = i X Z
    if (l == 'X') return map_local({q}, 1, 0, 0);
    if (l == 'Z') return map_local({q}, 0, 1, 0);
    return map_local({q}, 1, 1, 1);
  }

  void physical_gate(const std::string& g, int q0, int q1) {
    std::vector<int> qs = {q0};
    if (q1 >= 0) qs.push_back(q1);
    const ConjTable& t = conj_table(g, true);
    std::vector<Pauli> nimg;
    for (int j = 0; j < t.w; j++)
      for (int k = 0; k < 2; k++) {
        LocalPauli lp = t.img[2 * j + k];
        nimg.push_back(map_local(qs, lp.x, lp.z, lp.ph));
      }
    for (int j = 0; j < t.w; j++)
      for (int k = 0; k < 2; k++) img[2 * qs[j] + k] = nimg[2 * j + k];
  }

  // Conjugate a Pauli by a virtual gate (H, S on a; CX a->b; CZ a,b).
  static void vconj(Pauli& p, char g, int a, int b) {
    if (g == 'H') {
      bool xa = p.xb(a), za = p.zb(a);
      if (xa && za) p.ph = (p.ph + 2) & 3;
      p.setx(a, za);
      p.setz(a, xa);
    } else if (g == 'S') {
      bool xa = p.xb(a);
      if (xa) {
        p.ph = (p.ph + 1) & 3;
        p.setz(a, !p.zb(a));
      }
    } else if (g == 'C') {  // CX a -> b
      if (p.xb(a)) p.setx(b, !p.xb(b));
      if (p.zb(b)) p.setz(a, !p.zb(a));
    } else if (g == 'Z') {  // CZ
      bool xa = p.xb(a), xb = p.xb(b);
      if (xa && xb) p.ph = (p.ph + 2) & 3;
      if (xb) p.setz(a, !p.zb(a));
      if (xa) p.setz(b, !p.zb(b));
    }
  }

  void emit(const Op& o, std::vector<int64_t> uses = {}, int64_t def = -1) {
    flush_outputs_unless_noise(o.code);
    code.push_back({o, std::move(uses), def});
  }

  Op mk(uint8_t code_) {
    Op o;
    std::memset(&o, 0, sizeof(o));
    o.code = code_;
    return o;
  }

  // U_C <- U_C V^dagger for one virtual gate, and the matching bytecode.
  void virtual_gate(char g, int a, int b, Pauli* track) {
    for (auto& p : img) vconj(p, g, a, b);
    if (track) vconj(*track, g, a, b);
    bool a_act = pos_of[a] >= 0;
    bool b_act = b >= 0 && pos_of[b] >= 0;
    Op o = mk(0);
    o.a = (uint16_t)a;
    o.b = (uint16_t)(b >= 0 ? b : 0);
    o.pa = (uint8_t)(a_act ? pos_of[a] : 0);
    o.pb = (uint8_t)(b_act ? pos_of[b] : 0);
    bool on_state = (g == 'H' || g == 'S') ? a_act : (a_act && b_act);
    switch (g) {
      case 'H': o.code = on_state ? OP_ARRAY_H : OP_FRAME_H; break;
      case 'S': o.code = on_state ? OP_ARRAY_S : OP_FRAME_S; break;
      case 'C': o.code = on_state ? OP_ARRAY_CX : OP_FRAME_CX; break;
      case 'Z': o.code = on_state ? OP_ARRAY_CZ : OP_FRAME_CZ; break;
    }
    if (on_state) counts.array_ops++;
    emit(o);
  }

  // Lemma 1 / App. A with the dormant-first pivot. Returns v (or -1 for a
  // dormant Z string), sets kind ('X' / 'Z') and sign bit a.
  int localize(Pauli& p, char& kind, int& a) {
    if (!p.xzero()) {
      int v = -1, first = -1;
      for (int q = 0; q < n; q++)
        if (p.xb(q)) {
          if (first < 0) first = q;
          if (pos_of[q] < 0) { v = q; break; }
        }
      if (v < 0) v = first;
      std::vector<int> xs;
      for (int q = 0; q < n; q++)
        if (q != v && p.xb(q)) xs.push_back(q);
      if (pos_of[v] >= 0)
        for (int q : xs)
          if (pos_of[q] < 0) fail(9, "active pivot with dormant x-support");
      for (int q : xs) virtual_gate('C', v, q, &p);
      std::vector<int> zs;
      for (int q = 0; q < n; q++)
        if (q != v && p.zb(q)) zs.push_back(q);
      for (int q : zs) virtual_gate('Z', v, q, &p);
      if (p.zb(v)) virtual_gate('S', v, -1, &p);
      kind = 'X';
      a = herm_sign(p);
      return v;
    }
    int v = -1;
    for (int q = 0; q < n; q++)
      if (p.zb(q) && pos_of[q] >= 0) { v = q; break; }
    if (v < 0) return -1;
    std::vector<int> zs;
    for (int q = 0; q < n; q++)
      if (q != v && p.zb(q)) zs.push_back(q);
    for (int q : zs) virtual_gate('C', q, v, &p);
    kind = 'Z';
    a = herm_sign(p);
    return v;
  }

  uint32_t add_mask(const Pauli& p, bool with_x, bool with_z) {
    uint32_t off = (uint32_t)masks.size();
    auto put = [&](const std::vector<uint64_t>& v) {
      for (int w = 0; w < nw32; w++) masks.push_back((uint32_t)(v[w >> 1] >> (32 * (w & 1))));
    };
    if (with_x) put(p.x);
    if (with_z) put(p.z);
    return off;
  }

  void flush_outputs_unless_noise(uint8_t c) {
    if (c == OP_NOISE_BLOCK || c == OP_REC_OUT) return;
    flush_outputs();
  }
  void flush_outputs() {
    for (size_t i = 0; i < pending_out.size(); i++) {
      Op o = mk(OP_REC_OUT);
      o.i3 = (uint32_t)pending_row[i];
      code.push_back({o, {pending_out[i]}, -1});
    }
    pending_out.clear();
    pending_row.clear();
  }

  void noise_site(int64_t site, uint8_t kind, double p, uint32_t eff, int64_t flip_id) {
    if ((int64_t)site_p.size() != site) fail(9, "site numbering");
    site_p.push_back(p);
    site_kind.push_back(kind);
    site_eff.push_back(eff);
    site_flip_id.push_back(flip_id);
    if (!code.empty() && code.back().op.code == OP_NOISE_BLOCK && code.back().op.i1 == (uint32_t)site) {
      code.back().op.i1 = (uint32_t)site + 1;
      if (flip_id >= 0) code.back().uses.push_back(flip_id);
      return;
    }
    Op o = mk(OP_NOISE_BLOCK);
    o.i0 = (uint32_t)site;
    o.i1 = (uint32_t)site + 1;
    std::vector<int64_t> u;
    if (flip_id >= 0) u.push_back(flip_id);
    code.push_back({o, u, -1});
  }

  // Virtual masks of the K options of a noise site, each given as a Pauli of
  // the HIR frame.
  uint32_t noise_masks(const std::vector<Pauli>& opts) {
    uint32_t off = (uint32_t)masks.size();
    for (const Pauli& o : opts) add_mask(map_pauli(o), true, true);
    return off;
  }

  // exp(-i theta P) for P given in the HIR frame.
  void rotation(const Pauli& hp, double theta) {
    Pauli p = map_pauli(hp);
    char kind;
    int a;
    int v = localize(p, kind, a);
    if (v < 0) return;  // scalar phase on the dormant |0>
    double ta = a ? -theta : theta;
    if (kind == 'X' && pos_of[v] < 0) {
      virtual_gate('H', v, -1, nullptr);
      Op e = mk(OP_EXPAND_ROT);
      e.a = (uint16_t)v;
      e.pa = (uint8_t)act.size();
      e.f = ta;
      e.cs = std::cos(2.0 * ta);
      e.sn = std::sin(2.0 * ta);
      pos_of[v] = (int)act.size();
      act.push_back(v);
      k_max = std::max<uint32_t>(k_max, (uint32_t)act.size());
      if (act.size() > kMaxK) fail(3, "active dimension above the supported maximum");
      counts.array_ops++;
      emit(e);
    } else {
      Op r = mk(kind == 'Z' ? OP_ROT_Z : OP_ROT_X);
      r.a = (uint16_t)v;
      r.pa = (uint8_t)pos_of[v];
      r.f = ta;
      r.cs = kind == 'Z' ? std::cos(2.0 * ta) : std::cos(ta);
      r.sn = kind == 'Z' ? std::sin(2.0 * ta) : std::sin(ta);
      counts.array_ops++;
      emit(r);
    }
  }

  // Expectation-value probe (Sec. 3.2): M(P) for the product P; the frame
  // sign and the active-vector reduction are per shot (OP_EXPVAL).
  void probe(const Pauli& hp, int64_t index) {
    Pauli p = map_pauli(hp);
    Op e = mk(OP_EXPVAL);
    e.i0 = add_mask(p, true, true);
    e.i3 = (uint32_t)index;
    e.pa = (uint8_t)(p.ph & 3);
    for (int q = 0; q < n; q++) {
      if (pos_of[q] < 0) {
        if (p.xb(q)) e.pb = 1;  // x-support on a dormant qubit: <0|X|0> = 0
        continue;
      }
      if (p.xb(q)) e.i1 |= 1u << pos_of[q];
      if (p.zb(q)) e.i2 |= 1u << pos_of[q];
    }
    if (e.pb) e.i1 = e.i2 = 0;
    emit(e);
  }

  // Measurement of hp (HIR frame); a reset adds the conditional Pauli he.
  void measure(const PhysOp& o, const Pauli& hp, const Pauli& he) {
    Pauli p = map_pauli(hp);
    int64_t id = next_id++;
    bool active_z = false;
    for (int q = 0; q < n && !active_z; q++)
      if (p.zb(q) && pos_of[q] >= 0) active_z = true;
    // every record is written by its measurement; a later record-flip fault
    // patches the output bit (no separate output instruction)
    bool direct_out = o.record >= 0;
    if (p.xzero() && !active_z) {
      Op m = mk(OP_MEAS_STATIC);
      m.i0 = add_mask(p, false, true);
      m.i1 = (uint32_t)o.event;
      m.flags = (uint8_t)(herm_sign(p) ? FLAG_SIGN : 0);
      if (direct_out) { m.flags |= FLAG_OUT; m.i3 = (uint32_t)o.record; }
      counts.n_static++;
      emit(m, {}, id);
    } else {
      char kind;
      int a;
      int v = localize(p, kind, a);
      if (v < 0) fail(9, "measurement localisation failed");
      if (pos_of[v] < 0) {
        Op m = mk(OP_MEAS_RANDOM);
        m.a = (uint16_t)v;
        m.i0 = (uint32_t)o.event;
        m.i1 = (uint32_t)o.event;
        m.flags = (uint8_t)(a ? FLAG_SIGN : 0);
        if (direct_out) { m.flags |= FLAG_OUT; m.i3 = (uint32_t)o.record; }
        counts.n_random++;
        emit(m, {}, id);
        // the kernel applies H_v to the frame; mirror it in U_C
        for (auto& q : img) vconj(q, 'H', v, -1);
      } else {
        Op m = mk(kind == 'Z' ? OP_MEAS_ACTIVE_Z : OP_MEAS_ACTIVE_X);
        m.a = (uint16_t)v;
        m.pa = (uint8_t)pos_of[v];
        m.i0 = (uint32_t)o.event;
        m.i1 = (uint32_t)o.event;
        m.flags = (uint8_t)(a ? FLAG_SIGN : 0);
        if (direct_out) { m.flags |= FLAG_OUT; m.i3 = (uint32_t)o.record; }
        counts.n_active++;
        counts.array_ops++;
        emit(m, {}, id);
        int pos = pos_of[v];
        int top = act.back();
        act[pos] = top;
        pos_of[top] = pos;
        act.pop_back();
        pos_of[v] = -1;
        if (kind == 'X')
          for (auto& q : img) vconj(q, 'H', v, -1);
      }
    }
    if (o.reset) {
      Pauli e = map_pauli(he);
      Op f = mk(OP_FEEDFORWARD);
      f.i0 = add_mask(e, true, true);
      emit(f, {id}, -1);
    }
    if (o.record >= 0) {
      if (o.record >= (int64_t)record_id.size() || record_id[o.record] >= 0) fail(9, "record numbering");
      record_id[o.record] = id;
    }
  }
};

}  // namespace

// Store up to kInline u16 entries in the instruction (e[0..3], count in pa);
// entries past the count hold `pad` (an all-zero row for reads, a scratch
// row for writes).
void set_inline(Op& o, const std::vector<uint32_t>& v, uint32_t pad) {
  if (v.size() > kInline || pad > 0xFFFF) {
    o.pa = kNoInline;
    return;
  }
  for (uint32_t x : v)
    if (x > 0xFFFF) {
      o.pa = kNoInline;
      return;
    }
  o.pa = (uint8_t)v.size();
  o.f = 0.0;
  for (size_t i = 0; i < kInline; i++) o.e[i] = (uint16_t)(i < v.size() ? v[i] : pad);
}

Op mk_op(uint8_t code) {
  Op o;
  std::memset(&o, 0, sizeof(o));
  o.code = code;
  return o;
}

// Frame plane indices of a mask (x part then z part, nw words each).
std::vector<uint32_t> mask_planes(const std::vector<uint32_t>& masks, uint32_t off, uint32_t nw, uint32_t n,
                                  bool has_x, bool has_z) {
  std::vector<uint32_t> out;
  for (int part = 0; part < 2; part++) {
    if ((part == 0 && !has_x) || (part == 1 && !has_z)) continue;
    uint32_t base = off + ((part == 1 && has_x) ? nw : 0);
    for (uint32_t w = 0; w < nw; w++) {
      uint32_t bits = masks[base + w];
      while (bits) {
        uint32_t q = w * 32 + (uint32_t)__builtin_ctz(bits);
        bits &= bits - 1;
        out.push_back(part == 0 ? q : n + q);
      }
    }
  }
  return out;
}

// ---------------------------------------------------------------------------
// HIR (Sec. 3.1, stages 1-2): every active operation as a Pauli of the t = 0
// frame, P -> U^dagger P U with U the physical Cliffords before it (Def. 1).
// The back end localises the list in order; its U_C then holds only the
// localising Cliffords, and mapping through it gives the same Pauli as one
// walk through physical gates and localisations together, so an untouched
// list compiles to the same bytecode. Two operations commute iff their Paulis
// do (symplectic parity), which is all the passes below use.
// ---------------------------------------------------------------------------
namespace {

enum HKind : uint8_t { H_ROT, H_MEAS, H_FLIP, H_NOISE, H_FF, H_DET, H_OBS, H_PROBE };

struct Hir {
  HKind kind = H_ROT;
  uint32_t src = 0;         // physical operation (Flattener::ops index)
  Pauli p;                  // rotation axis, measured, feed-forward or probe Pauli
  Pauli e;                  // R / MR: the conditional X after the measurement
  std::vector<Pauli> opts;  // noise options
  double theta = 0.0;       // rotation exp(-i theta p)
  bool reset = false;
  int64_t rec = -1;         // record written (MEAS) or read (FLIP, FF)
  bool dead = false;
};

constexpr size_t kHirScan = 1u << 16;  // longest stretch a pass looks through

bool commute(const Pauli& a, const Pauli& b) {
  int c = 0;
  for (size_t w = 0; w < a.x.size(); w++) c += popc64((a.x[w] & b.z[w]) ^ (a.z[w] & b.x[w]));
  return (c & 1) == 0;
}

bool same_axis(const Pauli& a, const Pauli& b) { return a.x == b.x && a.z == b.z; }

// f on every Pauli through which h acts on the state (none for the
// classical operations); false as soon as f is.
template <class F>
bool each_pauli(const Hir& h, F f) {
  switch (h.kind) {
    case H_ROT: case H_FF: case H_PROBE: return f(h.p);
    case H_MEAS: return f(h.p) && (!h.reset || f(h.e));
    case H_NOISE:
      for (const Pauli& o : h.opts)
        if (!f(o)) return false;
      return true;
    default: return true;
  }
}

bool reads_record(const Hir& h, int64_t r, const std::vector<PhysOp>& ops) {
  if (r < 0) return false;
  if (h.kind == H_FLIP || h.kind == H_FF) return h.rec == r;
  if (h.kind == H_DET || h.kind == H_OBS) {
    const auto& rs = ops[h.src].recs;
    return std::find(rs.begin(), rs.end(), r) != rs.end();
  }
  return false;
}

// a and b, adjacent, may trade places without changing a probability, a
// state that is later observed, or a record.
bool swappable(const Hir& a, const Hir& b, const std::vector<PhysOp>& ops) {
  if (a.dead || b.dead) return true;
  // a probe reads the state where it stands
  if (a.kind == H_PROBE || b.kind == H_PROBE) return false;
  // noise sites keep their order (the survival sampler visits them so)
  const bool na = a.kind == H_NOISE || a.kind == H_FLIP, nb = b.kind == H_NOISE || b.kind == H_FLIP;
  if (na && nb) return false;
  // measurements keep their place among detectors: a shot rejected by
  // postselection has zero records after its failing detector
  // measurements keep their order: a draw is compared with the outcome's
  // probability given the outcomes before it, so two correlated commuting
  // measurements swapped give other records for the same draws
  const bool ma = a.kind == H_MEAS, mb = b.kind == H_MEAS;
  if (ma && mb) return false;
  if ((ma && (b.kind == H_DET || b.kind == H_OBS)) || (mb && (a.kind == H_DET || a.kind == H_OBS))) return false;
  if ((ma && reads_record(b, a.rec, ops)) || (mb && reads_record(a, b.rec, ops))) return false;
  return each_pauli(a, [&](const Pauli& pa) { return each_pauli(b, [&](const Pauli& pb) { return commute(pa, pb); }); });
}

// Phase fusion: a rotation about the axis of an earlier one, everything in
// between commuting with it, joins that one (angles add; opposite signs of
// the two Paulis subtract).
bool hir_fuse(std::vector<Hir>& L, const std::vector<PhysOp>& ops) {
  bool changed = false;
  for (size_t i = 0; i < L.size(); i++) {
    Hir& r = L[i];
    if (r.dead || r.kind != H_ROT) continue;
    size_t steps = 0;
    for (size_t j = i; j-- > 0 && steps < kHirScan;) {
      Hir& o = L[j];
      if (o.dead) continue;
      steps++;
      if (o.kind == H_ROT && same_axis(o.p, r.p)) {
        const int d = ((r.p.ph - o.p.ph) % 4 + 4) % 4;  // r.p = i^d o.p, d = 0 or 2
        o.theta += d == 0 ? r.theta : -r.theta;
        r.dead = true;
        changed = true;
        break;
      }
      if (!swappable(o, r, ops)) break;
    }
  }
  return changed;
}

// Q <- C^dagger Q C on every Pauli of h, C = exp(-i m pi/4 P), m = 1, 2, 3.
// For Q anticommuting with P, C^dagger Q C = exp(i m pi/2 P) Q: -Q for
// m = 2, -i Q P for m = 1 and i Q P for m = 3 (3 pi/4 = -pi/4 up to a global
// phase).
void hir_conjugate(Hir& h, const Pauli& P, int m) {
  auto f = [&](Pauli& q) {
    if (commute(q, P)) return;
    if (m == 2) {
      q.ph = (q.ph + 2) & 3;
      return;
    }
    pmul_inplace(q, P);
    q.ph = (q.ph + (m == 1 ? 3 : 1)) & 3;
  };
  switch (h.kind) {
    case H_ROT: case H_FF: case H_PROBE: f(h.p); break;
    case H_MEAS:
      f(h.p);
      if (h.reset) f(h.e);
      break;
    case H_NOISE:
      for (Pauli& o : h.opts) f(o);
      break;
    default: break;
  }
}

// Inverse cancellation and Clifford re-absorption: after fusion, a rotation
// whose angle is a multiple of pi/4 is a Clifford (pi/4), a Pauli (pi/2) or
// the identity (0, pi) up to a global phase. It is moved past every later
// operation, each conjugated by it, and then acts after the last record:
// it leaves the list.
bool hir_absorb_cliffords(std::vector<Hir>& L) {
  bool changed = false;
  for (size_t i = 0; i < L.size(); i++) {
    Hir& r = L[i];
    if (r.dead || r.kind != H_ROT) continue;
    const double q = r.theta / (M_PI / 4);
    const double m = std::nearbyint(q);
    if (std::fabs(q - m) > 1e-9 || std::fabs(m) > 1e9) continue;
    const int mm = (int)((((int64_t)m) % 4 + 4) % 4);
    r.dead = true;
    changed = true;
    if (mm == 0) continue;
    for (size_t j = i + 1; j < L.size(); j++)
      if (!L[j].dead) hir_conjugate(L[j], r.p, mm);
  }
  return changed;
}

// A rotation whose axis is measured later, everything in between commuting
// with it, acts just before that measurement on a state the projector then
// fixes: exp(-i theta P) Pi_m = e^{-+i theta} Pi_m, a phase per outcome
// branch. It is dropped.
bool hir_absorb_into_measurements(std::vector<Hir>& L, const std::vector<PhysOp>& ops) {
  bool changed = false;
  for (size_t i = 0; i < L.size(); i++) {
    Hir& r = L[i];
    if (r.dead || r.kind != H_ROT) continue;
    size_t steps = 0;
    for (size_t j = i + 1; j < L.size() && steps < kHirScan; j++) {
      const Hir& o = L[j];
      if (o.dead) continue;
      steps++;
      if (o.kind == H_MEAS && same_axis(o.p, r.p)) {
        r.dead = true;
        changed = true;
        break;
      }
      if (!swappable(r, o, ops)) break;
    }
  }
  return changed;
}

// Commuting reorder: measurements earlier, rotations later, so that the
// active dimension contracts before it grows. A measurement moves before the
// earliest rotation it can pass (every operation it passes commutes with
// it); a rotation moves after the last measurement it can pass. Nothing
// moves that would pass no such operation.
bool hir_reorder(std::vector<Hir>& L, const std::vector<PhysOp>& ops) {
  bool changed = false;
  L.erase(std::remove_if(L.begin(), L.end(), [](const Hir& h) { return h.dead; }), L.end());
  for (size_t i = 0; i < L.size(); i++) {
    if (L[i].kind != H_MEAS) continue;
    size_t best = i;
    for (size_t j = i, steps = 0; j-- > 0 && steps < kHirScan; steps++) {
      if (!swappable(L[j], L[i], ops)) break;
      if (L[j].kind == H_ROT) best = j;
    }
    if (best < i) {
      std::rotate(L.begin() + best, L.begin() + i, L.begin() + i + 1);
      changed = true;
    }
  }
  for (size_t i = L.size(); i-- > 0;) {
    if (L[i].kind != H_ROT) continue;
    size_t best = i;
    for (size_t j = i + 1, steps = 0; j < L.size() && steps < kHirScan; j++, steps++) {
      if (!swappable(L[i], L[j], ops)) break;
      if (L[j].kind == H_MEAS) best = j;
    }
    if (best > i) {
      std::rotate(L.begin() + i, L.begin() + i + 1, L.begin() + best + 1);
      changed = true;
    }
  }
  return changed;
}

}  // namespace

// ---------------------------------------------------------------------------
// Entry point
// ---------------------------------------------------------------------------
namespace {

// Array-traversal bytes per shot a program costs the batched executor: its
// whole count, less the shared noiseless prefix (run once per call, every
// shot then starts from one copy of its vector) where the executor takes it
// (at least 6 axes).
double per_shot_cost(const CompiledProgram& c) {
  const ProgHeader& h = *reinterpret_cast<const ProgHeader*>(c.blob.data());
  double b = c.counts.array_bytes;
  if (h.prefix_end > 0 && h.prefix_k >= 6) b -= c.counts.prefix_bytes - 8.0 * std::ldexp(1.0, (int)h.prefix_k);
  return b;
}
}  // namespace


namespace {
// The circuit up to its HIR, built once per nc_compile: the flattened
// operations and every active operation as a Pauli of the t = 0 frame.
struct Front {
  Flattener fl;
  std::vector<int64_t> flip_record;  // flip site -> its record
  std::vector<Hir> hir;
  bool any_rot = false;
};

int front_end(const std::string& text, Front& f, std::string& err) {
  try {
    std::vector<std::string> lines;
    {
      size_t s = 0;
      while (s <= text.size()) {
        size_t e = text.find('\n', s);
        std::string line = text.substr(s, e == std::string::npos ? std::string::npos : e - s);
        size_t hash = line.find('#');
        if (hash != std::string::npos) line = line.substr(0, hash);
        line = trim(line);
        if (!line.empty()) lines.push_back(line);
        if (e == std::string::npos) break;
        s = e + 1;
      }
    }
    size_t pos = 0;
    auto block = parse_lines(lines, pos, 0);
    Flattener& fl = f.fl;
    fl.run(block);

    // ---------------- front end: the HIR ----------------
    // Flip sites of one measurement instruction follow all of its
    // measurements (a flip changes only its record, never the frame, so
    // deferring it past the instruction's other targets is exact).
    // flip site -> its record
    std::vector<int64_t>& flip_record = f.flip_record;
    flip_record.assign(fl.site_p.size(), -1);
    for (auto& po : fl.ops)
      if (po.kind == K_MEAS && po.site >= 0) flip_record[po.site] = po.record;
    std::vector<Hir>& hir = f.hir;
    {
      Compiler fe((int)fl.n_q);  // physical Cliffords only: img = U^dagger P U
      const int nw = fe.nw64;
      std::vector<Hir> flips;
      int cur_instr = -2;
      auto letter_of = [](const PhysOp& o) {
        return o.name == "T" || o.name == "T_DAG" ? 'Z' : o.name.back();
      };
      for (size_t pi = 0; pi < fl.ops.size(); pi++) {
        const PhysOp& po = fl.ops[pi];
        if (!(po.kind == K_MEAS && po.instr == cur_instr)) {
          for (auto& f : flips) hir.push_back(std::move(f));
          flips.clear();
        }
        cur_instr = po.kind == K_MEAS ? po.instr : -2;
        Hir h;
        h.src = (uint32_t)pi;
        h.p = Pauli(nw);
        switch (po.kind) {
          case K_GATE:
            fe.physical_gate(po.name, po.q0, po.q1);
            continue;
          case K_ROT:
            h.kind = H_ROT;
            h.p = fe.map_letter(po.q0, letter_of(po));
            h.theta = po.name == "T" ? M_PI / 8 : po.name == "T_DAG" ? -M_PI / 8 : po.arg / 2.0;
            break;
          case K_MEAS:
            h.kind = H_MEAS;
            h.p = fe.map_letter(po.q0, po.xbasis ? 'X' : 'Z');
            h.reset = po.reset;
            if (po.reset) h.e = fe.map_letter(po.q0, 'X');
            h.rec = po.record;
            if (po.record >= 0 && po.site >= 0) {
              Hir f;
              f.kind = H_FLIP;
              f.src = (uint32_t)pi;
              f.rec = po.record;
              flips.push_back(std::move(f));
            }
            break;
          case K_NOISE: {
            h.kind = H_NOISE;
            static const char* letters = "IXYZ";
            auto opt = [&](char la, char lb) {
              Pauli acc(nw);
              if (la != 'I') pmul_inplace(acc, fe.map_letter(po.q0, la));
              if (lb != 'I') pmul_inplace(acc, fe.map_letter(po.q1, lb));
              h.opts.push_back(acc);
            };
            switch (fl.site_kind[po.site]) {
              case SITE_X: opt('X', 'I'); break;
              case SITE_Y: opt('Y', 'I'); break;
              case SITE_Z: opt('Z', 'I'); break;
              case SITE_D1: opt('X', 'I'); opt('Y', 'I'); opt('Z', 'I'); break;
              case SITE_D2:
                for (int j = 1; j < 16; j++) opt(letters[j >> 2], letters[j & 3]);
                break;
            }
            break;
          }
          case K_FF:
            h.kind = H_FF;
            h.p = fe.map_letter(po.q0, po.name[0]);
            h.rec = po.recs[0];
            break;
          case K_DET: h.kind = H_DET; break;
          case K_OBS: h.kind = H_OBS; break;
          case K_PROBE:
            h.kind = H_PROBE;
            for (size_t j = 0; j < po.recs.size(); j++) pmul_inplace(h.p, fe.map_letter((int)po.recs[j], po.name[j]));
            break;
        }
        hir.push_back(std::move(h));
      }
      for (auto& f : flips) hir.push_back(std::move(f));
    }

    for (const Hir& h : hir) f.any_rot |= h.kind == H_ROT;
    return 0;
  } catch (CompileError& e) {
    err = e.what();
    return e.code;
  } catch (std::bad_alloc&) {
    err = "out of host memory";
    return 6;
  } catch (std::exception& e) {
    err = e.what();
    return 9;
  }
}

// The HIR passes the flags leave on, in their order (Sec. 3.1, stage 2):
// fusion and re-absorption to a fixed point, the peephole, the reorder.
// Returns the kNoFuse / kNoPeephole / kNoReorder bits of the passes that
// changed the list.
uint32_t run_passes(std::vector<Hir>& hir, const std::vector<PhysOp>& ops, uint32_t flags) {
  uint32_t changed = 0;
  if (!(flags & kNoFuse))
    for (int it = 0; it < 4; it++) {
      const bool a = hir_fuse(hir, ops);
      const bool b = hir_absorb_cliffords(hir);
      if (!a && !b) break;
      changed |= kNoFuse;
    }
  if (!(flags & kNoPeephole) && hir_absorb_into_measurements(hir, ops)) changed |= kNoPeephole;
  if (!(flags & kNoReorder) && hir_reorder(hir, ops)) changed |= kNoReorder;
  return changed;
}

// Localisation, bytecode and tables of one HIR list.
int back_end(const Front& f, const std::vector<Hir>& hir, CompiledProgram& out, std::string& err) {
  try {
    const Flattener& fl = f.fl;
    const std::vector<int64_t>& flip_record = f.flip_record;
    // ---------------- back end: localisation and bytecode ----------------
    Compiler c((int)fl.n_q);
    c.record_id.assign((size_t)fl.rec, -1);
    int64_t kept_id = -1;
    std::vector<int64_t> obs_id(fl.n_obs, -1);
    for (const Hir& h : hir) {
      if (h.dead) continue;
      const PhysOp& po = fl.ops[h.src];
      switch (h.kind) {
        case H_ROT:
          c.rotation(h.p, h.theta);
          break;
        case H_MEAS:
          c.measure(po, h.p, h.e);
          break;
        case H_FLIP:
          c.noise_site(po.site, SITE_FLIP, fl.site_p[po.site], 0, c.record_id[po.record]);
          break;
        case H_NOISE: {
          uint32_t eff = c.noise_masks(h.opts);
          c.noise_site(po.site, fl.site_kind[po.site], po.arg, eff, -1);
          break;
        }
        case H_FF: {
          Op f = c.mk(OP_FEEDFORWARD);
          f.i0 = c.add_mask(c.map_pauli(h.p), true, true);
          c.emit(f, {c.record_id[po.recs[0]]}, -1);
          break;
        }
        case H_DET: {
          Op d = c.mk(OP_DETECTOR);
          d.i3 = (uint32_t)po.index;
          std::vector<int64_t> u;
          for (auto r : po.recs) u.push_back(c.record_id[r]);
          d.i1 = (uint32_t)u.size();
          c.emit(d, u, -1);
          break;
        }
        case H_PROBE:
          c.probe(h.p, po.index);
          break;
        case H_OBS: {
          if (obs_id[po.index] < 0) obs_id[po.index] = c.next_id++;
          Op d = c.mk(OP_OBS_INCLUDE);
          std::vector<int64_t> u;
          for (auto r : po.recs) u.push_back(c.record_id[r]);
          d.i1 = (uint32_t)u.size();
          d.i2 = (uint32_t)obs_id[po.index];  // id, rewritten to a slot below
          c.emit(d, u, -1);
          break;
        }
      }
    }
    c.flush_outputs();
    // observables never included still get an (all-zero) accumulator
    for (int64_t o = 0; o < fl.n_obs; o++)
      if (obs_id[o] < 0) obs_id[o] = c.next_id++;
    for (int64_t o = 0; o < fl.n_obs; o++) {
      Op d = c.mk(OP_OBS_OUT);
      d.i3 = (uint32_t)o;
      c.code.push_back({d, {}, -1});
    }
    kept_id = c.next_id++;
    {
      Op d = c.mk(OP_KEPT_OUT);
      c.code.push_back({d, {}, -1});
    }
    c.code.push_back({c.mk(OP_END), {}, -1});

    // ---------------- fuse static resets with their conditional X ----------------
    {
      std::vector<int64_t> n_uses(c.next_id, 0);
      for (auto& e : c.code)
        for (auto id : e.uses) n_uses[id]++;
      std::vector<Emitted> fused;
      fused.reserve(c.code.size());
      for (size_t i = 0; i < c.code.size(); i++) {
        Emitted& e = c.code[i];
        if (e.op.code == OP_MEAS_STATIC && !(e.op.flags & FLAG_OUT) && e.def >= 0 && i + 1 < c.code.size() &&
            c.code[i + 1].op.code == OP_FEEDFORWARD && c.code[i + 1].uses.size() == 1 &&
            c.code[i + 1].uses[0] == e.def && n_uses[e.def] == 1) {
          auto mp = mask_planes(c.masks, e.op.i0, (uint32_t)c.nw32, (uint32_t)c.n, true, false);
          auto ep = mask_planes(c.masks, c.code[i + 1].op.i0, (uint32_t)c.nw32, (uint32_t)c.n, true, true);
          if (mp.size() <= kInline && ep.size() <= 4 && 2 * (uint32_t)c.n + 1 <= 0xFFFF) {
            Op o = e.op;
            set_inline(o, mp, 2 * (uint32_t)c.n);
            o.flags |= FLAG_RESET;
            o.pb = (uint8_t)ep.size();
            for (int j = 0; j < 4; j++) o.r[j] = j < (int)ep.size() ? (uint16_t)ep[j] : (uint16_t)(2 * c.n + 1);
            fused.push_back({o, {}, -1});
            i++;
            continue;
          }
        }
        fused.push_back(e);
      }
      c.code.swap(fused);
    }

    // ---------------- record-slot allocation (linear scan) ----------------
    int64_t n_ids = c.next_id;
    std::vector<int64_t> last_use(n_ids, -1);
    std::vector<char> persistent(n_ids, 0);
    persistent[kept_id] = 1;
    for (auto id : obs_id) persistent[id] = 1;
    for (size_t i = 0; i < c.code.size(); i++) {
      for (auto id : c.code[i].uses) last_use[id] = (int64_t)i;
      if (c.code[i].def >= 0) last_use[c.code[i].def] = std::max<int64_t>(last_use[c.code[i].def], (int64_t)i);
    }
    std::vector<int64_t> slot_of(n_ids, -1);
    std::vector<uint32_t> free_slots;
    uint32_t n_slots = 0;
    auto alloc = [&]() -> uint32_t {
      if (!free_slots.empty()) {
        uint32_t s = free_slots.back();
        free_slots.pop_back();
        return s;
      }
      return n_slots++;
    };
    slot_of[kept_id] = alloc();
    for (auto id : obs_id) slot_of[id] = alloc();
    std::vector<uint32_t> slot_list;
    std::vector<Op> ops;
    ops.reserve(c.code.size());
    for (size_t i = 0; i < c.code.size(); i++) {
      Emitted& e = c.code[i];
      if (e.def >= 0) slot_of[e.def] = alloc();
      Op o = e.op;
      switch (o.code) {
        case OP_MEAS_STATIC:
          if (o.flags & FLAG_RESET) break;
          o.i2 = (uint32_t)slot_of[e.def];
          // the mask is the z-support of the mapped observable; the parity
          // reads the frame's x planes on that support
          set_inline(o, mask_planes(c.masks, o.i0, (uint32_t)c.nw32, (uint32_t)c.n, true, false), 2 * (uint32_t)c.n);
          break;
        case OP_MEAS_RANDOM: case OP_MEAS_ACTIVE_Z: case OP_MEAS_ACTIVE_X:
          o.i2 = (uint32_t)slot_of[e.def];
          break;
        case OP_FEEDFORWARD:
          o.i2 = (uint32_t)slot_of[e.uses[0]];
          set_inline(o, mask_planes(c.masks, o.i0, (uint32_t)c.nw32, (uint32_t)c.n, true, true), 2 * (uint32_t)c.n + 1);
          break;
        case OP_REC_OUT:
          o.i2 = (uint32_t)slot_of[e.uses[0]];
          break;
        case OP_DETECTOR:
        case OP_OBS_INCLUDE: {
          o.i0 = (uint32_t)slot_list.size();
          std::vector<uint32_t> sl;
          for (auto id : e.uses) sl.push_back((uint32_t)slot_of[id]);
          slot_list.insert(slot_list.end(), sl.begin(), sl.end());
          if (o.code == OP_OBS_INCLUDE) o.i2 = (uint32_t)slot_of[o.i2];
          set_inline(o, sl, 0);  // re-padded below with the zero slot row, once n_slots is known
          break;
        }
        case OP_OBS_OUT:
          o.i2 = (uint32_t)slot_of[obs_id[o.i3]];
          break;
        case OP_KEPT_OUT:
          o.i2 = (uint32_t)slot_of[kept_id];
          break;
        default:
          break;
      }
      ops.push_back(o);
      // free ids whose last use is this op
      std::vector<int64_t> touched = e.uses;
      if (e.def >= 0) touched.push_back(e.def);
      std::sort(touched.begin(), touched.end());
      touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
      for (auto id : touched)
        if (!persistent[id] && last_use[id] == (int64_t)i && slot_of[id] >= 0) {
          free_slots.push_back((uint32_t)slot_of[id]);
        }
    }
    // slot lists: pad with the zero slot row (index n_slots), or give up inlining
    for (auto& o : ops)
      if ((o.code == OP_DETECTOR || o.code == OP_OBS_INCLUDE) && o.pa != kNoInline) {
        if (n_slots > 0xFFFF) {
          o.pa = kNoInline;
          continue;
        }
        for (uint32_t i = o.pa; i < kInline; i++) o.e[i] = (uint16_t)n_slots;
      }

    // batch runs of independent list instructions (Sec. 3.1 stage 4: cut
    // dispatch; here also to give the executor independent loads to overlap)
    {
      auto kind_of = [&](const Op& o) -> int {
        if (o.code == OP_MEAS_STATIC && o.pa != kNoInline) return (o.flags & FLAG_RESET) ? 2 : 1;
        if (o.code == OP_DETECTOR && o.pa != kNoInline) return 3;
        return 0;
      };
      const uint32_t trash = 2 * (uint32_t)c.n + 1;
      auto writes = [&](const Op& o, std::vector<uint32_t>& w) {
        w.clear();
        for (int j = 0; j < (int)o.pb; j++) w.push_back(o.r[j]);
      };
      auto reads = [&](const Op& o, std::vector<uint32_t>& r) {
        r.clear();
        for (uint32_t j = 0; j < o.pa; j++) r.push_back(o.e[j]);
        for (int j = 0; j < (int)o.pb; j++) r.push_back(o.r[j]);
      };
      std::vector<Op> out;
      out.reserve(ops.size() + ops.size() / 4);
      size_t i = 0;
      std::vector<uint32_t> wi, rj, wj;
      while (i < ops.size()) {
        const int kd = kind_of(ops[i]);
        size_t n = 1;
        if (kd) {
          std::vector<uint32_t> written;  // planes written by earlier members (resets)
          if (kd == 2) writes(ops[i], written);
          while (i + n < ops.size() && n < kMaxBatch && kind_of(ops[i + n]) == kd) {
            if (kd == 2) {
              reads(ops[i + n], rj);
              writes(ops[i + n], wj);
              bool clash = false;
              for (auto x : rj)
                if (x != trash && std::find(written.begin(), written.end(), x) != written.end()) clash = true;
              if (clash) break;
              written.insert(written.end(), wj.begin(), wj.end());
            }
            n++;
          }
          // header + n payloads must stay inside one staging chunk
          const size_t room = kChunk - (out.size() % kChunk);
          if (n + 1 > room) n = room > 1 ? room - 1 : 0;
        }
        if (kd && n >= 2) {
          Op hdr = mk_op(OP_BATCH);
          hdr.a = (uint16_t)kd;
          hdr.pa = (uint8_t)n;
          out.push_back(hdr);
          for (size_t u = 0; u < n; u++) out.push_back(ops[i + u]);
          i += n;
        } else {
          out.push_back(ops[i]);
          i++;
        }
      }
      ops.swap(out);
    }

    // noise-block ordinals and the site -> block table
    std::vector<uint32_t> site_blk(c.site_kind.size(), 0);
    uint32_t n_blocks = 0;
    for (auto& o : ops)
      if (o.code == OP_NOISE_BLOCK) {
        o.i2 = n_blocks;
        for (uint32_t s = o.i0; s < o.i1; s++) site_blk[s] = n_blocks;
        n_blocks++;
      }

    // flip sites reference slots through site_eff
    std::vector<uint32_t> site_eff = c.site_eff;
    for (size_t s = 0; s < c.site_kind.size(); s++)
      if (c.site_kind[s] == SITE_FLIP) site_eff[s] = (uint32_t)slot_of[c.site_flip_id[s]];
    // A flip slot must still be live at its noise block: it is, because the
    // block is a use of the id (recorded in Emitted::uses).

    // ---------------- sparse noise options ----------------
    std::vector<uint32_t> site_opt(c.site_kind.size(), 0), opt_tab;
    std::vector<uint16_t> plist;
    for (size_t s = 0; s < c.site_kind.size(); s++) {
      if (c.site_kind[s] == SITE_FLIP) {
        site_opt[s] = (uint32_t)(opt_tab.size() / 2);
        opt_tab.push_back(site_eff[s]);
        opt_tab.push_back((uint32_t)flip_record[s]);
        continue;
      }
      uint32_t k = c.site_kind[s] == SITE_D1 ? 3 : c.site_kind[s] == SITE_D2 ? 15 : 1;
      site_opt[s] = (uint32_t)(opt_tab.size() / 2);
      for (uint32_t j = 0; j < k; j++) {
        auto pl = mask_planes(c.masks, c.site_eff[s] + j * 2 * (uint32_t)c.nw32, (uint32_t)c.nw32,
                              (uint32_t)c.n, true, true);
        opt_tab.push_back((uint32_t)plist.size());
        opt_tab.push_back((uint32_t)pl.size());
        for (auto x : pl) plist.push_back((uint16_t)x);
      }
    }

    // ---------------- option records (site, option) -> 16 bytes ----------------
    std::vector<uint16_t> orec((size_t)c.site_kind.size() * kRecPerSite * 8, 0);
    for (size_t s = 0; s < c.site_kind.size(); s++) {
      const uint32_t k = c.site_kind[s] == SITE_D1 ? 3 : c.site_kind[s] == SITE_D2 ? 15 : 1;
      for (uint32_t j = 0; j < k; j++) {
        uint16_t* r = &orec[(s * kRecPerSite + j) * 8];
        const uint32_t oi = 2 * (site_opt[s] + (c.site_kind[s] == SITE_FLIP ? 0 : j));
        if (c.site_kind[s] == SITE_FLIP) {
          const uint32_t slot = opt_tab[oi], row = opt_tab[oi + 1];
          r[0] = kRecFlip;
          r[1] = (uint16_t)slot;
          r[2] = (uint16_t)(slot >> 16);
          r[3] = (uint16_t)row;
          r[4] = (uint16_t)(row >> 16);
        } else if (opt_tab[oi + 1] <= 7) {
          r[0] = (uint16_t)opt_tab[oi + 1];
          for (uint32_t e = 0; e < opt_tab[oi + 1]; e++) r[1 + e] = plist[opt_tab[oi] + e];
        } else {
          r[0] = kRecLong;
        }
      }
    }

    // ---------------- survival table (Sec. 3.2, integer form) ----------------
    size_t S = c.site_p.size();
    std::vector<uint64_t> q(S);
    std::vector<uint32_t> seg_start(S), seg_end(S), info(S);
    {
      size_t start = 0;
      double run = 1.0;
      std::vector<std::pair<size_t, size_t>> bounds;
      for (size_t i = 0; i < S; i++) {
        double p = c.site_p[i];
        double nxt = run * (1.0 - p);
        if (nxt < 1.0 / 65536.0 && i > start) {
          bounds.push_back({start, i});
          start = i;
          nxt = 1.0 * (1.0 - p);
        }
        run = nxt;
        q[i] = run >= 1.0 ? ~0ull : (uint64_t)(run * 18446744073709551616.0);
      }
      bounds.push_back({start, S});
      for (auto& b : bounds)
        for (size_t i = b.first; i < b.second; i++) {
          seg_start[i] = (uint32_t)b.first;
          seg_end[i] = (uint32_t)b.second;
        }
      for (size_t i = 0; i < S; i++) {
        uint32_t k = c.site_kind[i] == SITE_D1 ? 3 : c.site_kind[i] == SITE_D2 ? 15 : 1;
        uint32_t idx = site_opt[i];
        if (idx >= (1u << 24)) fail(2, "noise option table too large");
        info[i] = (uint32_t)c.site_kind[i] | (k << 4) | (idx << 8);
      }
    }

    // ---------------- survival search records and guide tables ----------------
    std::vector<SrchRec> srch(S);
    std::vector<uint32_t> guide;
    for (size_t a = 0; a < S;) {
      const size_t b = seg_end[a];
      // smallest shift with at most max(16, 2 (b - a)) buckets
      const uint64_t target = std::max<uint64_t>(16, 2 * (uint64_t)(b - a));
      uint32_t shift = 0;
      while (((uint64_t)guide_key(q[b - 1], shift) + 1) > target) shift++;
      const uint32_t base = (uint32_t)guide.size(), m = guide_key(q[b - 1], shift) + 1;
      // g[j] = first site i of the segment with key(Q[i]) >= j
      size_t i = a;
      for (uint32_t j = 0; j < m; j++) {
        while (i < b - 1 && guide_key(q[i], shift) < j) i++;
        guide.push_back((uint32_t)i);
      }
      for (size_t st = a; st < b; st++) {
        SrchRec& r = srch[st];
        r.a = (uint32_t)a;
        r.b = (uint32_t)b;
        r.gbase = base;
        r.shift = shift;
        r.q_end = q[b - 1];
        r.q_l = st == a ? ~0ull : q[st - 1];
      }
      a = b;
    }

    // ---------------- blob ----------------
    ProgHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kMagic;
    h.version = kVersion;
    h.n_qubits = (uint32_t)c.n;
    h.nw = (uint32_t)c.nw32;
    h.n_ops = (uint32_t)ops.size();
    h.n_sites = (uint32_t)S;
    h.n_meas = (uint32_t)fl.rec;
    h.n_det = (uint32_t)fl.det;
    h.n_obs = (uint32_t)fl.n_obs;
    h.n_events = (uint32_t)fl.ev;
    h.n_slots = n_slots;
    h.k_max = c.k_max;
    h.kept_slot = (uint32_t)slot_of[kept_id];
    h.n_mask_words = (uint32_t)c.masks.size();
    h.n_slot_list = (uint32_t)slot_list.size();
    h.n_opt = (uint32_t)(opt_tab.size() / 2);
    h.n_plist = (uint32_t)plist.size();
    h.n_blocks = n_blocks;
    h.n_guide = (uint32_t)guide.size();
    h.n_probes = (uint32_t)fl.probe;
    {
      // shared prefix: frame, array and rotation instructions from the start
      uint32_t k = 0, pe = 0;
      for (; pe < ops.size(); pe++) {
        const uint8_t cd = ops[pe].code;
        if (!(cd >= OP_FRAME_H && cd <= OP_ROT_X)) break;
        if (cd == OP_EXPAND_ROT) k++;
      }
      h.prefix_end = pe;
      h.prefix_k = k;
    }
    {
      double mean = 0.0;
      for (double sp : c.site_p) mean += sp;
      h.mean_faults = (float)mean;
    }
    uint64_t off = (sizeof(ProgHeader) + 15) & ~15ull;
    auto place = [&](uint64_t bytes) {
      uint64_t o = off;
      off = (off + bytes + 15) & ~15ull;
      return o;
    };
    h.off_ops = place(ops.size() * sizeof(Op));
    h.off_masks = place(c.masks.size() * 4);
    h.off_q = place(S * 8);
    h.off_seg_start = place(S * 4);
    h.off_seg_end = place(S * 4);
    h.off_site_info = place(S * 4);
    h.off_site_eff = place(S * 4);
    h.off_slot_list = place(slot_list.size() * 4);
    h.off_det_ref = place((size_t)fl.det * 4);
    h.off_obs_ref = place((size_t)fl.n_obs * 4);
    h.off_site_opt = place(S * 4);
    h.off_opt_tab = place(opt_tab.size() * 4);
    h.off_plist = place(plist.size() * 2);
    h.off_orec = place(orec.size() * 2);
    h.off_site_blk = place(site_blk.size() * 4);
    h.off_srch = place(S * sizeof(SrchRec));
    h.off_guide = place(guide.size() * 4);
    h.off_site_p = place(S * 8);
    h.total_bytes = off;
    out.blob.assign(off, 0);
    std::memcpy(out.blob.data(), &h, sizeof(h));
    auto cp = [&](uint64_t o, const void* src, size_t bytes) {
      if (bytes) std::memcpy(out.blob.data() + o, src, bytes);
    };
    cp(h.off_ops, ops.data(), ops.size() * sizeof(Op));
    cp(h.off_masks, c.masks.data(), c.masks.size() * 4);
    cp(h.off_q, q.data(), S * 8);
    cp(h.off_seg_start, seg_start.data(), S * 4);
    cp(h.off_seg_end, seg_end.data(), S * 4);
    cp(h.off_site_info, info.data(), S * 4);
    cp(h.off_site_eff, site_eff.data(), S * 4);
    cp(h.off_slot_list, slot_list.data(), slot_list.size() * 4);
    cp(h.off_site_opt, site_opt.data(), S * 4);
    cp(h.off_opt_tab, opt_tab.data(), opt_tab.size() * 4);
    cp(h.off_plist, plist.data(), plist.size() * 2);
    cp(h.off_orec, orec.data(), orec.size() * 2);
    cp(h.off_site_blk, site_blk.data(), site_blk.size() * 4);
    cp(h.off_srch, srch.data(), S * sizeof(SrchRec));
    cp(h.off_guide, guide.data(), guide.size() * 4);
    cp(h.off_site_p, c.site_p.data(), S * 8);
    append_affine(out.blob);
    append_fused(out.blob);
    {
      // array traffic of one shot through the (unfused) instruction list
      double bytes = 0.0;
      uint32_t k = 0;
      ProgHeader hh;
      std::memcpy(&hh, out.blob.data(), sizeof(hh));
      for (size_t pc = 0; pc < ops.size(); pc++) {
        if (pc == hh.prefix_end) c.counts.prefix_bytes = bytes;
        const Op& o = ops[pc];
        const double dim = std::ldexp(1.0, (int)k);
        switch (o.code) {
          case OP_EXPAND_ROT: bytes += 8.0 * 3.0 * dim; k++; break;
          case OP_ARRAY_H: case OP_ARRAY_S: case OP_ARRAY_CX: case OP_ARRAY_CZ: case OP_ROT_Z: case OP_ROT_X:
            bytes += 8.0 * 2.0 * dim;
            break;
          case OP_MEAS_ACTIVE_Z: case OP_MEAS_ACTIVE_X: bytes += 8.0 * 2.5 * dim; k--; break;
          default: break;
        }
      }
      c.counts.array_bytes = bytes;
    }
    out.counts = c.counts;
    return 0;
  } catch (CompileError& e) {
    err = e.what();
    return e.code;
  } catch (std::bad_alloc&) {
    err = "out of host memory";
    return 6;
  } catch (std::exception& e) {
    err = e.what();
    return 9;
  }
}
}  // namespace

int compile_program(const std::string& text, uint32_t flags, CompiledProgram& out, std::string& err) {
  // The HIR passes never change a record, but they can raise the per-shot
  // cost: the reorder pulls measurements ahead of rotations, which can end
  // the shared noiseless prefix sooner, and a re-absorbed Clifford can turn
  // later measured Paulis into ones whose localisation takes more array
  // instructions. The front end runs once; the program with every pass the
  // flags leave on is compiled first, then each subset of the passes that
  // changed the list there (dropping passes that changed nothing gives the
  // same list), and the cheapest per shot is kept, the one with more passes
  // on a tie. Programs without rotations compile once.
  Front f;
  int rc = front_end(text, f, err);
  if (rc != 0) return rc;
  if (!f.any_rot) return back_end(f, f.hir, out, err);
  CompiledProgram best;
  double best_cost = 0.0;
  int first_rc = -1;
  std::string first_err;
  auto consider = [&](const std::vector<Hir>& L) -> int {
    CompiledProgram c;
    std::string e;
    const int r = back_end(f, L, c, e);
    if (first_rc < 0) {
      first_rc = r;
      first_err = e;
    }
    if (r == 3) return 0;  // over the active-dimension limit with these passes
    if (r != 0) {
      err = e;
      return r;
    }
    const double cost = per_shot_cost(c);
    if (best.blob.empty() || cost < best_cost) {
      best_cost = cost;
      best = std::move(c);
    }
    return 0;
  };
  uint32_t active = 0;
  {
    std::vector<Hir> all = f.hir;
    active = run_passes(all, f.fl.ops, flags);
    rc = consider(all);
    if (rc != 0) return rc;
  }
  const bool zero_k = !best.blob.empty() && reinterpret_cast<const ProgHeader*>(best.blob.data())->k_max == 0;
  for (uint32_t off = 1; off <= kNoPeephole + kNoReorder + kNoFuse && !zero_k; off++) {
    if (off & ~active) continue;  // only passes that changed the list are varied
    std::vector<Hir> L = f.hir;
    run_passes(L, f.fl.ops, flags | off);
    rc = consider(L);
    if (rc != 0) return rc;
  }
  if (best.blob.empty()) {
    err = first_err;
    return first_rc;
  }
  out = std::move(best);
  return 0;
}

}  // namespace nc
