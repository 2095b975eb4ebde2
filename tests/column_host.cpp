// Host driver for the column arithmetic of the CUDA library (mw_column.cuh),
// compiled as plain C++ by tests/test_column_host.py and compared there with
// the oracle.  One request per input line, one answer line per request:
//   cut W S F m x_0 .. x_{m-1}    (x_j as 16 hex digits of the double's bits)
//     -> "ok|range d_0 .. d_{S-1}"   balanced digits, d_0 most significant
//   round m ex n u_0 .. u_{n-1}   (u_i 32-bit limbs, least significant first,
//                                  two's complement, as 8 hex digits)
//     -> "w_0 .. w_{m-1}"            greedy words as 16 hex digits of their bits
//   bf16 d                        -> the bfloat16 bits of the integer d (4 hex digits)
//   fuse g n D s_0 .. s_{D-1}     (int32 diagonal sums, s_0 most significant)
//     -> "u_0 .. u_{n-1} | v_0 .. v_{n-1}"  X = sum_t s_t 2^(8 (D-1-t)) in n 32-bit
//        limbs by fuse_w8 and by fuse_diagonals with groups of g (two's complement)
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <iostream>
#include <sstream>
#include <string>
#include <vector>

#include "mw_column.cuh"
#include "mw_fuse.cuh"

using namespace mw;

static double bits_to_double(uint64_t b) {
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
}
static uint64_t double_to_bits(double x) {
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
}

template <int MW, int W>
static std::string cut(int S, int F, const std::vector<double> &w) {
  double x[MW];
  for (int j = 0; j < MW; ++j) x[j] = w[j];
  std::vector<uint32_t> col(cut_column_slots(W, S), 0u);
  std::vector<int32_t> d(S, 0);
  const bool ok = cut_column<MW, W>(x, F, S, col.data(), 1,
                                    [&](int k, int32_t v) { d[S - 1 - k] = v; });
  for (uint32_t v : col)
    if (v != 0) return "column-not-zero";
  std::ostringstream o;
  o << (ok ? "ok" : "range");
  for (int p = 0; p < S; ++p) o << ' ' << d[p];
  return o.str();
}

template <int MW>
static std::string cut_m(int W, int S, int F, const std::vector<double> &w) {
  return W == 8 ? cut<MW, 8>(S, F, w) : cut<MW, 24>(S, F, w);
}

template <int MW, int NL32>
static std::string round_n(int ex, const std::vector<uint32_t> &u) {
  uint32_t U[NL32];
  for (int i = 0; i < NL32; ++i) U[i] = i < (int)u.size() ? u[i] : 0u;
  std::vector<uint32_t> col(NL32, 0u);
  double out[MW];
  round_column<MW, NL32>(U, col.data(), 1, ex, [&](int k, double v) { out[k] = v; });
  std::ostringstream o;
  for (int k = 0; k < MW; ++k) {
    char buf[24];
    std::snprintf(buf, sizeof buf, "%016llx", (unsigned long long)double_to_bits(out[k]));
    o << (k ? " " : "") << buf;
  }
  return o.str();
}

template <int MW>
static std::string round_m(int ex, int n, const std::vector<uint32_t> &u) {
  switch (n) {
    case 8: return round_n<MW, 8>(ex, u);
    case 12: return round_n<MW, 12>(ex, u);
    case 20: return round_n<MW, 20>(ex, u);
    case 34: return round_n<MW, 34>(ex, u);
  }
  return "bad-limbs";
}

template <int NL32>
static std::string fuse_n(int g, const std::vector<int32_t> &sv) {
  const int D = (int)sv.size();
  uint32_t U[NL32];
  fuse_w8<NL32>(U, sv.data(), 1, D);
  uint64_t X[NL32 / 2];
  for (int i = 0; i < NL32 / 2; ++i) X[i] = 0;
  fuse_diagonals<NL32 / 2>(X, sv.data(), 1, D, g, 8);
  uint32_t V[NL32];
  to_limbs32<NL32 / 2>(X, V);
  std::ostringstream o;
  char buf[16];
  for (int i = 0; i < NL32; ++i) {
    std::snprintf(buf, sizeof buf, "%08x", U[i]);
    o << (i ? " " : "") << buf;
  }
  o << " |";
  for (int i = 0; i < NL32; ++i) {
    std::snprintf(buf, sizeof buf, "%08x", V[i]);
    o << ' ' << buf;
  }
  return o.str();
}

int main() {
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string op;
    in >> op;
    if (op == "cut") {
      int W, S, F, m;
      in >> W >> S >> F >> m;
      std::vector<double> w(m);
      for (int j = 0; j < m; ++j) {
        std::string h;
        in >> h;
        w[j] = bits_to_double(std::stoull(h, nullptr, 16));
      }
      std::string r = "bad-m";
      if (m == 2) r = cut_m<2>(W, S, F, w);
      if (m == 4) r = cut_m<4>(W, S, F, w);
      if (m == 8) r = cut_m<8>(W, S, F, w);
      if (m == 16) r = cut_m<16>(W, S, F, w);
      std::cout << r << '\n';
    } else if (op == "round") {
      int m, ex, n;
      in >> m >> ex >> n;
      std::vector<uint32_t> u(n);
      for (int i = 0; i < n; ++i) {
        std::string h;
        in >> h;
        u[i] = (uint32_t)std::stoul(h, nullptr, 16);
      }
      std::string r = "bad-m";
      if (m == 2) r = round_m<2>(ex, n, u);
      if (m == 4) r = round_m<4>(ex, n, u);
      if (m == 8) r = round_m<8>(ex, n, u);
      if (m == 16) r = round_m<16>(ex, n, u);
      std::cout << r << '\n';
    } else if (op == "fuse") {
      int g, n, D;
      in >> g >> n >> D;
      std::vector<int32_t> sv(D);
      for (int t = 0; t < D; ++t) in >> sv[t];
      std::string r = "bad-limbs";
      if (n == 10) r = fuse_n<10>(g, sv);
      if (n == 18) r = fuse_n<18>(g, sv);
      if (n == 20) r = fuse_n<20>(g, sv);
      std::cout << r << '\n';
    } else if (op == "bf16") {
      int d;
      in >> d;
      char buf[8];
      std::snprintf(buf, sizeof buf, "%04x", (unsigned)small_int_bf16(d));
      std::cout << buf << '\n';
    } else {
      std::cout << "bad-op\n";
    }
  }
  return 0;
}
