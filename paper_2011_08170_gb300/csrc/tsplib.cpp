// TSPLIB reader (host): the input of the GD program of Section 5.1 is the 2-D
// coordinates of the nodes in TSPLIB format.
//
// Accepted: the keyword part (NAME, COMMENT, TYPE, DIMENSION, EDGE_WEIGHT_TYPE,
// ... as "KEY : value" or "KEY value" lines), then NODE_COORD_SECTION with one
// "id x y" line per node, ids 1..DIMENSION each once in any order, then
// optionally EOF.  EDGE_WEIGHT_TYPE must be EUC_2D (the nearest-integer
// Euclidean length this library computes) and TYPE, if given, TSP.  The
// library works on integer coordinates in [0, 2^20): every coordinate must be
// integral (written as 12, 12.0 or 1.2e1), and the points are translated so
// that the smallest x and the smallest y become 0 (lengths do not change); the
// translation is returned.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/f2m.h"

namespace {

thread_local std::string g_tsp_error;

f2m_status tsp_fail(const std::string& m) {
  g_tsp_error = m;
  return F2M_ERR_INVALID_ARG;
}

std::string upper(std::string s) {
  for (char& ch : s) ch = (char)std::toupper((unsigned char)ch);
  return s;
}

std::string trim(const std::string& s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

}  // namespace

extern "C" const char* f2m_tsplib_last_error(void) { return g_tsp_error.c_str(); }

extern "C" f2m_status f2m_tsplib_parse(const char* text, int64_t len, int32_t* xy, int32_t cap,
                                       int32_t* n_out, int64_t* translation) {
  g_tsp_error.clear();
  if (!text || len < 0 || !n_out) return tsp_fail("NULL argument");
  *n_out = 0;
  int64_t dim = -1;
  bool in_coords = false, euc = false;
  std::vector<double> px, py;
  std::vector<char> seen;
  int64_t got = 0;
  int64_t pos = 0, lineno = 0;
  while (pos < len) {
    int64_t end = pos;
    while (end < len && text[end] != '\n') ++end;
    std::string line = trim(std::string(text + pos, (size_t)(end - pos)));
    pos = end + 1;
    ++lineno;
    if (line.empty()) continue;
    const std::string up = upper(line);
    if (up == "EOF") break;
    if (!in_coords) {
      if (up == "NODE_COORD_SECTION") {
        if (!euc) return tsp_fail("EDGE_WEIGHT_TYPE EUC_2D must come before NODE_COORD_SECTION");
        if (dim < 1) return tsp_fail("DIMENSION must come before NODE_COORD_SECTION");
        in_coords = true;
        continue;
      }
      size_t k = 0;
      while (k < line.size() && line[k] != ':' && !std::isspace((unsigned char)line[k])) ++k;
      const std::string key = upper(line.substr(0, k));
      std::string val = trim(line.substr(k));
      if (!val.empty() && val[0] == ':') val = trim(val.substr(1));
      const std::string uval = upper(val);
      if (key == "DIMENSION") {
        char* e = nullptr;
        const long long d = std::strtoll(val.c_str(), &e, 10);
        if (e == val.c_str() || d < 1 || d >= (1LL << 24)) return tsp_fail("DIMENSION must be in [1, 2^24)");
        dim = d;
        px.assign((size_t)d, 0.0);
        py.assign((size_t)d, 0.0);
        seen.assign((size_t)d, 0);
      } else if (key == "EDGE_WEIGHT_TYPE") {
        if (uval != "EUC_2D") return tsp_fail("EDGE_WEIGHT_TYPE " + val + " is not supported (EUC_2D only)");
        euc = true;
      } else if (key == "TYPE") {
        if (uval != "TSP") return tsp_fail("TYPE " + val + " is not supported (TSP only)");
      } else if (key.find("SECTION") != std::string::npos) {
        return tsp_fail("section " + key + " is not supported (NODE_COORD_SECTION only)");
      }
      continue;  // NAME, COMMENT and other keywords are ignored
    }
    // "id x y"
    const char* s = line.c_str();
    char* e = nullptr;
    const long long id = std::strtoll(s, &e, 10);
    if (e == s) return tsp_fail("line " + std::to_string(lineno) + ": node id expected");
    s = e;
    const double x = std::strtod(s, &e);
    if (e == s) return tsp_fail("line " + std::to_string(lineno) + ": x expected");
    s = e;
    const double y = std::strtod(s, &e);
    if (e == s) return tsp_fail("line " + std::to_string(lineno) + ": y expected");
    if (id < 1 || id > dim) return tsp_fail("line " + std::to_string(lineno) + ": node id out of 1..DIMENSION");
    if (seen[(size_t)(id - 1)]) return tsp_fail("line " + std::to_string(lineno) + ": node id repeated");
    if (!std::isfinite(x) || !std::isfinite(y) || x != std::floor(x) || y != std::floor(y))
      return tsp_fail("line " + std::to_string(lineno) + ": coordinates must be integral");
    seen[(size_t)(id - 1)] = 1;
    px[(size_t)(id - 1)] = x;
    py[(size_t)(id - 1)] = y;
    ++got;
  }
  if (!in_coords) return tsp_fail("no NODE_COORD_SECTION");
  if (got != dim) return tsp_fail("NODE_COORD_SECTION has " + std::to_string(got) + " nodes, DIMENSION " + std::to_string(dim));
  double mx = px[0], my = py[0], Mx = px[0], My = py[0];
  for (int64_t i = 1; i < dim; ++i) {
    mx = std::fmin(mx, px[(size_t)i]);
    my = std::fmin(my, py[(size_t)i]);
    Mx = std::fmax(Mx, px[(size_t)i]);
    My = std::fmax(My, py[(size_t)i]);
  }
  if (Mx - mx >= (double)(1 << 20) || My - my >= (double)(1 << 20))
    return tsp_fail("coordinate spread must be below 2^20 in x and in y");
  *n_out = (int32_t)dim;
  if (translation) {
    translation[0] = (int64_t)mx;
    translation[1] = (int64_t)my;
  }
  if (!xy) return F2M_OK;  // size query
  if (cap < dim) return tsp_fail("xy buffer holds fewer than DIMENSION points");
  for (int64_t i = 0; i < dim; ++i) {
    xy[2 * i] = (int32_t)(px[(size_t)i] - mx);
    xy[2 * i + 1] = (int32_t)(py[(size_t)i] - my);
  }
  return F2M_OK;
}
