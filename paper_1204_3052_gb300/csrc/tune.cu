// Tile table of a plan: launch shapes per precision and range of orders
// (the paper picks its product kernel's tile shape by problem size and local
// memory, arXiv 1204.3052 Sec. 4.3.7; here an autotuner measures the
// candidates and these rules carry its choices).  Host code only: a small
// JSON reader for the table file, validation, lookup and the plan hooks.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "plan.h"

using namespace mp;

namespace {

// ---- JSON: objects, arrays, strings, numbers, true / false / null -----------

struct Reader {
  const char* s;
  const char* p;
  std::string err;

  void ws() {
    while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p;
  }
  bool fail(const char* what) {
    if (err.empty()) {
      char b[160];
      snprintf(b, sizeof b, "%s at offset %ld", what, (long)(p - s));
      err = b;
    }
    return false;
  }
  bool lit(const char* w) {
    const size_t n = strlen(w);
    if (strncmp(p, w, n) != 0) return fail("unexpected token");
    p += n;
    return true;
  }
  bool str(std::string* out) {
    ws();
    if (*p != '"') return fail("expected a string");
    ++p;
    out->clear();
    while (*p && *p != '"') {
      if (*p == '\\') {
        ++p;
        if (!*p) break;
        if (*p == 'u') {  // keys and values here are ASCII; keep the escape as '?'
          for (int k = 0; k < 5 && *p; ++k) ++p;
          out->push_back('?');
          continue;
        }
        const char c = *p == 'n' ? '\n' : *p == 't' ? '\t' : *p;
        out->push_back(c);
        ++p;
        continue;
      }
      out->push_back(*p++);
    }
    if (*p != '"') return fail("unterminated string");
    ++p;
    return true;
  }
  bool num(double* out) {
    ws();
    char* end = nullptr;
    errno = 0;
    const double v = strtod(p, &end);
    if (end == p || errno == ERANGE) return fail("expected a number");
    p = end;
    *out = v;
    return true;
  }
  // Skip any value.
  bool skip(int depth = 0) {
    ws();
    if (depth > 64) return fail("nesting too deep");
    if (*p == '{' || *p == '[') {
      const char close = *p == '{' ? '}' : ']';
      const bool obj = *p == '{';
      ++p;
      ws();
      if (*p == close) {
        ++p;
        return true;
      }
      for (;;) {
        if (obj) {
          std::string k;
          if (!str(&k)) return false;
          ws();
          if (*p != ':') return fail("expected ':'");
          ++p;
        }
        if (!skip(depth + 1)) return false;
        ws();
        if (*p == ',') {
          ++p;
          continue;
        }
        if (*p == close) {
          ++p;
          return true;
        }
        return fail("expected ',' or a closing bracket");
      }
    }
    if (*p == '"') {
      std::string t;
      return str(&t);
    }
    if (*p == 't') return lit("true");
    if (*p == 'f') return lit("false");
    if (*p == 'n') return lit("null");
    double d;
    return num(&d);
  }
};

int precision_code(const std::string& s) {
  if (s == "fp32" || s == "fp32_simt") return MATPOW_FP32_SIMT;
  if (s == "bf16") return MATPOW_BF16;
  if (s == "bf16x3") return MATPOW_BF16X3;
  if (s == "bf16x6") return MATPOW_BF16X6;
  return -1;
}

// One rule object; unknown keys are skipped.
bool read_rule(Reader& r, matpow_tile_rule* out) {
  *out = matpow_tile_rule{-1, -1, -1, -1, -1, -1, -1};
  r.ws();
  if (*r.p != '{') return r.fail("expected a rule object");
  ++r.p;
  r.ws();
  if (*r.p == '}') {
    ++r.p;
    return true;
  }
  for (;;) {
    std::string k;
    if (!r.str(&k)) return false;
    r.ws();
    if (*r.p != ':') return r.fail("expected ':'");
    ++r.p;
    r.ws();
    int* field = k == "n_lo" ? &out->n_lo : k == "n_hi" ? &out->n_hi : k == "bn" ? &out->bn
               : k == "split_k" ? &out->split_k : k == "chain" ? &out->chain
               : k == "persist" ? &out->persist : nullptr;
    if (k == "precision") {
      if (*r.p == '"') {
        std::string v;
        if (!r.str(&v)) return false;
        out->precision = precision_code(v);
        if (out->precision < 0) return r.fail("unknown precision");
      } else {
        double d;
        if (!r.num(&d)) return false;
        out->precision = (int)d;
      }
    } else if (field) {
      if (*r.p == 'n') {
        if (!r.lit("null")) return false;
        *field = -1;
      } else {
        double d;
        if (!r.num(&d)) return false;
        if (d != (double)(int)d) return r.fail("expected an integer");
        *field = (int)d;
      }
    } else if (!r.skip()) {
      return false;
    }
    r.ws();
    if (*r.p == ',') {
      ++r.p;
      continue;
    }
    if (*r.p == '}') {
      ++r.p;
      return true;
    }
    return r.fail("expected ',' or '}'");
  }
}

bool parse_table(const char* json, std::vector<matpow_tile_rule>* rules, std::string* err) {
  Reader r{json, json, {}};
  rules->clear();
  bool seen = false;
  r.ws();
  if (*r.p != '{') {
    *err = "tile table: expected a JSON object at offset 0";
    return false;
  }
  ++r.p;
  r.ws();
  if (*r.p != '}') {
    for (;;) {
      std::string k;
      if (!r.str(&k)) break;
      r.ws();
      if (*r.p != ':') {
        r.fail("expected ':'");
        break;
      }
      ++r.p;
      if (k == "rules") {
        seen = true;
        r.ws();
        if (*r.p != '[') {
          r.fail("expected the rules array");
          break;
        }
        ++r.p;
        r.ws();
        if (*r.p == ']') {
          ++r.p;
        } else {
          bool ok = true;
          for (;;) {
            matpow_tile_rule t;
            if (!read_rule(r, &t)) {
              ok = false;
              break;
            }
            rules->push_back(t);
            r.ws();
            if (*r.p == ',') {
              ++r.p;
              continue;
            }
            if (*r.p == ']') {
              ++r.p;
              break;
            }
            r.fail("expected ',' or ']'");
            ok = false;
            break;
          }
          if (!ok) break;
        }
      } else if (!r.skip()) {
        break;
      }
      r.ws();
      if (*r.p == ',') {
        ++r.p;
        continue;
      }
      if (*r.p == '}') {
        ++r.p;
        break;
      }
      r.fail("expected ',' or '}'");
      break;
    }
  } else {
    ++r.p;
  }
  if (r.err.empty()) {
    r.ws();
    if (*r.p) r.fail("trailing text");
  }
  if (r.err.empty() && !seen) r.err = "no \"rules\" array";
  if (!r.err.empty()) {
    *err = "tile table: " + r.err;
    return false;
  }
  return true;
}

bool valid_rule(const matpow_tile_rule& t, std::string* why) {
  char b[200];
  if (t.precision < MATPOW_FP32_SIMT || t.precision > MATPOW_BF16X6) {
    snprintf(b, sizeof b, "unknown precision %d", t.precision);
  } else if (t.n_lo < 0 || t.n_hi <= t.n_lo) {
    snprintf(b, sizeof b, "order range (%d, %d] is empty", t.n_lo, t.n_hi);
  } else if (t.bn != -1 && t.bn != 64 && t.bn != 128) {
    snprintf(b, sizeof b, "bn=%d (64, 128 or -1)", t.bn);
  } else if (t.split_k != -1 && t.split_k != 1 && t.split_k != 2 && t.split_k != 4) {
    snprintf(b, sizeof b, "split_k=%d (1, 2, 4 or -1)", t.split_k);
  } else if (t.chain < -1 || t.chain > 1 || t.persist < -1 || t.persist > 1) {
    snprintf(b, sizeof b, "chain=%d persist=%d (0, 1 or -1)", t.chain, t.persist);
  } else {
    return true;
  }
  *why = b;
  return false;
}

}  // namespace

const matpow_tile_rule* mp::plan_tile_rule(const matpow_plan_s* p, int N) {
  const matpow_tile_rule* hit = nullptr;
  for (const auto& t : p->tiles)
    if (t.precision == (int)p->prec && N > t.n_lo && N <= t.n_hi) hit = &t;
  return hit;
}

int mp::plan_tile_field(const matpow_plan_s* p, int N, int matpow_tile_rule::*field) {
  const matpow_tile_rule* t = plan_tile_rule(p, N);
  return t ? t->*field : -1;
}

extern "C" matpow_status matpow_tile_table_parse(const char* json, matpow_tile_rule* rules, int cap,
                                                 int* count) {
  if (!json || !count || cap < 0 || (cap > 0 && !rules))
    return fail(nullptr, MATPOW_EINVAL, "matpow_tile_table_parse: bad arguments");
  std::vector<matpow_tile_rule> v;
  std::string err;
  if (!parse_table(json, &v, &err)) return fail(nullptr, MATPOW_EINVAL, "%s", err.c_str());
  *count = (int)v.size();
  for (int i = 0; i < (int)v.size() && i < cap; ++i) rules[i] = v[i];
  return MATPOW_OK;
}

extern "C" matpow_status matpow_tile_rule_lookup(const matpow_tile_rule* rules, int count,
                                                 matpow_precision precision, int N, matpow_tile_rule* out) {
  if (!out || count < 0 || (count > 0 && !rules))
    return fail(nullptr, MATPOW_EINVAL, "matpow_tile_rule_lookup: bad arguments");
  const matpow_tile_rule* hit = nullptr;
  for (int i = 0; i < count; ++i)
    if (rules[i].precision == (int)precision && N > rules[i].n_lo && N <= rules[i].n_hi) hit = &rules[i];
  if (!hit) {
    *out = matpow_tile_rule{-1, -1, (int)precision, -1, -1, -1, -1};
    return MATPOW_EAGAIN;
  }
  *out = *hit;
  return MATPOW_OK;
}

extern "C" matpow_status matpow_plan_set_tile_table(matpow_plan_t p, const matpow_tile_rule* rules, int count) {
  if (!p) return fail(nullptr, MATPOW_EINVAL, "matpow_plan_set_tile_table: plan is NULL");
  if (count < 0 || (count > 0 && !rules))
    return fail(p, MATPOW_EINVAL, "matpow_plan_set_tile_table: bad arguments");
  for (int i = 0; i < count; ++i) {
    std::string why;
    if (!valid_rule(rules[i], &why))
      return fail(p, MATPOW_EINVAL, "matpow_plan_set_tile_table: rule %d: %s", i, why.c_str());
  }
  p->tiles.assign(rules, rules + count);
  drop_plan_graphs(p);  // cached graphs were captured with the old shapes
  if (p->batch.exec) {
    cudaGraphExecDestroy(p->batch.exec);
    p->batch.exec = nullptr;
    p->batch.sig.clear();
  }
  return MATPOW_OK;
}

extern "C" matpow_status matpow_plan_load_tile_table(matpow_plan_t p, const char* path) {
  if (!p || !path) return fail(p, MATPOW_EINVAL, "matpow_plan_load_tile_table: NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(p, MATPOW_EINVAL, "matpow_plan_load_tile_table: cannot open %s", path);
  std::string text;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) {
    text.append(buf, k);
    if (text.size() > (16u << 20)) {
      fclose(f);
      return fail(p, MATPOW_EINVAL, "matpow_plan_load_tile_table: %s is larger than 16 MiB", path);
    }
  }
  fclose(f);
  std::vector<matpow_tile_rule> v;
  std::string err;
  if (!parse_table(text.c_str(), &v, &err))
    return fail(p, MATPOW_EINVAL, "%s (%s)", err.c_str(), path);
  return matpow_plan_set_tile_table(p, v.data(), (int)v.size());
}
