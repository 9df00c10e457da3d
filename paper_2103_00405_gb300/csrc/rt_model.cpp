// rt_model.cpp -- the text model format of the paper's Table 4 (host side).
//
// A model file has an "# init" section of initial counts ("NAME = count"), a
// "# reactions" section with one reaction per line ("coef NAME coef NAME --> coef NAME : rate",
// NULL for no species, a coefficient of 1 may be left out), and after "# end" settings of the
// form "key = value" (the paper's "time" and "steps").  Lines starting with "//" are comments.
// Species are numbered in order of first appearance (init section first).  The parser returns
// the network in the COO form rt_network_create takes (reactant coefficients and net state
// changes, duplicates merged, zero net changes dropped), the rates, the initial state and the
// settings.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "rt_internal.h"

using namespace rt;

namespace {

std::string trim(const std::string &s) {
  size_t b = 0, e = s.size();
  while (b < e && std::isspace((unsigned char)s[b])) ++b;
  while (e > b && std::isspace((unsigned char)s[e - 1])) --e;
  return s.substr(b, e - b);
}

bool parse_int(const std::string &t, long long &v) {
  if (t.empty()) return false;
  char *end = nullptr;
  v = std::strtoll(t.c_str(), &end, 10);
  return end && *end == '\0';
}

bool parse_double(const std::string &t, double &v) {
  if (t.empty()) return false;
  char *end = nullptr;
  v = std::strtod(t.c_str(), &end);
  return end && *end == '\0' && std::isfinite(v);
}

bool valid_name(const std::string &t) {
  if (t.empty() || !(std::isalpha((unsigned char)t[0]) || t[0] == '_')) return false;
  for (char ch : t)
    if (!(std::isalnum((unsigned char)ch) || ch == '_' || ch == '.')) return false;
  return true;
}

struct Parsed {
  std::vector<std::string> names;
  std::map<std::string, int> index;
  std::vector<long long> x0;
  std::vector<std::map<int, int>> reac, prod;
  std::vector<double> c;
  double time = NAN;
  long long steps = -1;

  int species(const std::string &nm) {
    auto it = index.find(nm);
    if (it != index.end()) return it->second;
    const int id = (int)names.size();
    names.push_back(nm);
    index[nm] = id;
    x0.push_back(0);
    return id;
  }
};

// one side of a reaction: "NULL", or coefficient / name tokens
bool parse_side(Parsed &P, const std::string &side, std::map<int, int> &out, std::string &err) {
  std::istringstream is(side);
  std::vector<std::string> tok;
  for (std::string t; is >> t;) tok.push_back(t);
  if (tok.size() == 1 && (tok[0] == "NULL" || tok[0] == "null" || tok[0] == "0")) return true;
  if (tok.empty()) {
    err = "empty side (write NULL for no species)";
    return false;
  }
  long long coef = 1;
  bool have_coef = false;
  for (const std::string &t : tok) {
    long long v;
    if (parse_int(t, v)) {
      if (have_coef || v <= 0) {
        err = "bad coefficient '" + t + "'";
        return false;
      }
      coef = v;
      have_coef = true;
    } else if (t == "+") {
      continue;
    } else if (valid_name(t) && t != "NULL") {
      if (coef > 1000000) {
        err = "coefficient too large";
        return false;
      }
      out[P.species(t)] += (int)coef;
      coef = 1;
      have_coef = false;
    } else {
      err = "unexpected token '" + t + "'";
      return false;
    }
  }
  if (have_coef) {
    err = "coefficient without a species";
    return false;
  }
  return true;
}

}  // namespace

extern "C" int rt_model_parse(const char *text, rt_model **out) {
  clear_error();
  if (!out) return set_error(RT_ERR_INVALID_ARG, "rt_model_parse: out is NULL");
  *out = nullptr;
  if (!text) return set_error(RT_ERR_INVALID_ARG, "rt_model_parse: text is NULL");
  Parsed P;
  enum { NONE, INIT, REACTIONS, END } sec = NONE;
  std::istringstream in(text);
  std::string raw;
  int lineno = 0;
  while (std::getline(in, raw)) {
    ++lineno;
    std::string line = trim(raw);
    const size_t cpos = line.find("//");
    if (cpos != std::string::npos) line = trim(line.substr(0, cpos));
    if (line.empty()) continue;
    if (line[0] == '#') {
      const std::string h = trim(line.substr(1));
      if (h == "init") sec = INIT;
      else if (h == "reactions") sec = REACTIONS;
      else if (h == "end") sec = END;
      else return set_error(RT_ERR_INVALID_ARG, "line %d: unknown section '%s'", lineno, h.c_str());
      continue;
    }
    if (sec == INIT || sec == END) {
      const size_t eq = line.find('=');
      if (eq == std::string::npos)
        return set_error(RT_ERR_INVALID_ARG, "line %d: expected 'name = value'", lineno);
      const std::string key = trim(line.substr(0, eq)), val = trim(line.substr(eq + 1));
      if (sec == INIT) {
        long long v;
        if (!valid_name(key)) return set_error(RT_ERR_INVALID_ARG, "line %d: bad species name '%s'", lineno, key.c_str());
        if (!parse_int(val, v) || v < 0 || v > INT32_MAX)
          return set_error(RT_ERR_INVALID_ARG, "line %d: initial count must be an integer in [0, 2^31)", lineno);
        if (P.index.count(key)) return set_error(RT_ERR_INVALID_ARG, "line %d: species '%s' initialised twice", lineno, key.c_str());
        P.x0[P.species(key)] = v;
      } else {
        double v;
        if (!parse_double(val, v)) return set_error(RT_ERR_INVALID_ARG, "line %d: bad value '%s'", lineno, val.c_str());
        if (key == "time") P.time = v;
        else if (key == "steps") {
          if (v < 0 || v != std::floor(v)) return set_error(RT_ERR_INVALID_ARG, "line %d: steps must be a count", lineno);
          P.steps = (long long)v;
        }  // other settings are accepted and ignored
      }
      continue;
    }
    if (sec != REACTIONS) return set_error(RT_ERR_INVALID_ARG, "line %d: text outside a section", lineno);
    size_t arrow = line.find("-->");
    size_t alen = 3;
    if (arrow == std::string::npos) {
      arrow = line.find("->");
      alen = 2;
    }
    const size_t colon = line.rfind(':');
    if (arrow == std::string::npos || colon == std::string::npos || colon < arrow)
      return set_error(RT_ERR_INVALID_ARG, "line %d: expected 'reactants --> products : rate'", lineno);
    double rate;
    if (!parse_double(trim(line.substr(colon + 1)), rate) || rate < 0)
      return set_error(RT_ERR_INVALID_ARG, "line %d: rate must be a finite number >= 0", lineno);
    std::map<int, int> r, p;
    std::string err;
    if (!parse_side(P, line.substr(0, arrow), r, err) ||
        !parse_side(P, line.substr(arrow + alen, colon - arrow - alen), p, err))
      return set_error(RT_ERR_INVALID_ARG, "line %d: %s", lineno, err.c_str());
    P.reac.push_back(r);
    P.prod.push_back(p);
    P.c.push_back(rate);
  }
  if (P.c.empty()) return set_error(RT_ERR_INVALID_ARG, "no reactions");

  rt_model *m = new rt_model();
  const int N = (int)P.names.size(), M = (int)P.c.size();
  m->n_species = N;
  m->n_reactions = M;
  std::vector<int32_t> rr, rs, rc, sr, ss, sd;
  for (int k = 0; k < M; k++) {
    for (auto &e : P.reac[k]) {
      rr.push_back(k);
      rs.push_back(e.first);
      rc.push_back(e.second);
    }
    std::map<int, long long> d;
    for (auto &e : P.reac[k]) d[e.first] -= e.second;
    for (auto &e : P.prod[k]) d[e.first] += e.second;
    for (auto &e : d)
      if (e.second != 0) {
        sr.push_back(k);
        ss.push_back(e.first);
        sd.push_back((int32_t)e.second);
      }
  }
  auto copy_i32 = [](const std::vector<int32_t> &v) {
    int32_t *p = (int32_t *)std::malloc(sizeof(int32_t) * (v.size() ? v.size() : 1));
    if (!v.empty()) std::memcpy(p, v.data(), sizeof(int32_t) * v.size());
    return p;
  };
  m->n_reac_nz = (int64_t)rr.size();
  m->reac_rxn = copy_i32(rr);
  m->reac_sp = copy_i32(rs);
  m->reac_coef = copy_i32(rc);
  m->n_stoi_nz = (int64_t)sr.size();
  m->stoi_rxn = copy_i32(sr);
  m->stoi_sp = copy_i32(ss);
  m->stoi_delta = copy_i32(sd);
  m->c = (double *)std::malloc(sizeof(double) * M);
  std::memcpy(m->c, P.c.data(), sizeof(double) * M);
  m->x0 = (int32_t *)std::malloc(sizeof(int32_t) * (N ? N : 1));
  for (int i = 0; i < N; i++) m->x0[i] = (int32_t)P.x0[i];
  m->species_names = (char **)std::malloc(sizeof(char *) * (N ? N : 1));
  for (int i = 0; i < N; i++) {
    m->species_names[i] = (char *)std::malloc(P.names[i].size() + 1);
    std::memcpy(m->species_names[i], P.names[i].c_str(), P.names[i].size() + 1);
  }
  m->time = P.time;
  m->steps = P.steps;
  *out = m;
  return RT_OK;
}

extern "C" void rt_model_free(rt_model *m) {
  if (!m) return;
  std::free(m->reac_rxn);
  std::free(m->reac_sp);
  std::free(m->reac_coef);
  std::free(m->stoi_rxn);
  std::free(m->stoi_sp);
  std::free(m->stoi_delta);
  std::free(m->c);
  std::free(m->x0);
  for (int i = 0; i < m->n_species; i++) std::free(m->species_names[i]);
  std::free(m->species_names);
  delete m;
}
