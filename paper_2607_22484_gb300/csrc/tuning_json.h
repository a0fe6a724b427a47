// The autotune cache as JSON text (svt_tuning_export / svt_tuning_import).
//
//   {"format": 1, "gpu": "<device name>", "sms": <SM count>, "entries": [
//     {"m": .., "n": .., "iters": .., "prec": .., "schedule": .., "norm": .., "polish": ..,
//      "mode": .., "hp_steps": .., "ell0": .., "delta": .., "fuse": .., "widths": [..]}, ..]}
//
// Pure host code: a writer for that one layout and a small recursive-descent reader
// of JSON values (objects, arrays, numbers, strings, true/false/null), so that text a
// user edits or another tool writes is read strictly and rejected when malformed.
#pragma once

#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "plan.h"

namespace svt {

constexpr int kTuningFormat = 1;

inline std::string json_escape(const char *s)
{
    std::string o;
    for (; *s; ++s) {
        const unsigned char c = (unsigned char)*s;
        if (c == '"' || c == '\\') {
            o += '\\';
            o += (char)c;
        } else if (c < 0x20) {
            char b[8];
            std::snprintf(b, sizeof(b), "\\u%04x", c);
            o += b;
        } else {
            o += (char)c;
        }
    }
    return o;
}

inline std::string tuning_to_json(const char *gpu, int sms,
                                  const std::map<TuneKey, std::vector<int>> &tuning)
{
    std::string o = "{\"format\": " + std::to_string(kTuningFormat) + ", \"gpu\": \"" +
                    json_escape(gpu) + "\", \"sms\": " + std::to_string(sms) + ", \"entries\": [";
    bool first = true;
    char num[64];
    for (const auto &kv : tuning) {
        const TuneKey &k = kv.first;
        o += first ? "\n  {" : ",\n  {";
        first = false;
        o += "\"m\": " + std::to_string(k.m) + ", \"n\": " + std::to_string(k.n) +
             ", \"iters\": " + std::to_string(k.iters) + ", \"prec\": " + std::to_string(k.prec) +
             ", \"schedule\": " + std::to_string(k.schedule) + ", \"norm\": " +
             std::to_string(k.norm) + ", \"polish\": " + std::to_string(k.polish) +
             ", \"mode\": " + std::to_string(k.mode) + ", \"hp_steps\": " +
             std::to_string(k.hp_steps);
        std::snprintf(num, sizeof(num), "%.17g", k.ell0);
        o += std::string(", \"ell0\": ") + num;
        std::snprintf(num, sizeof(num), "%.17g", k.delta);
        o += std::string(", \"delta\": ") + num;
        o += ", \"fuse\": " + std::to_string(k.fuse) + ", \"widths\": [";
        for (size_t i = 0; i < kv.second.size(); ++i)
            o += (i ? ", " : "") + std::to_string(kv.second[i]);
        o += "]}";
    }
    o += first ? "]}\n" : "\n]}\n";
    return o;
}

// ---------------------------------------------------------------- reader

struct JVal {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0.0;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
    const JVal *get(const char *key) const
    {
        for (const auto &kv : obj)
            if (kv.first == key)
                return &kv.second;
        return nullptr;
    }
};

struct JReader {
    const char *p;
    int depth = 0;
    void ws()
    {
        while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')
            ++p;
    }
    bool lit(const char *w)
    {
        const size_t n = std::strlen(w);
        if (std::strncmp(p, w, n) != 0)
            return false;
        p += n;
        return true;
    }
    bool string(std::string &out)
    {
        if (*p != '"')
            return false;
        ++p;
        while (*p && *p != '"') {
            if ((unsigned char)*p < 0x20)
                return false;
            if (*p == '\\') {
                ++p;
                switch (*p) {
                case '"': out += '"'; break;
                case '\\': out += '\\'; break;
                case '/': out += '/'; break;
                case 'b': out += '\b'; break;
                case 'f': out += '\f'; break;
                case 'n': out += '\n'; break;
                case 'r': out += '\r'; break;
                case 't': out += '\t'; break;
                case 'u': {
                    unsigned v = 0;
                    for (int i = 1; i <= 4; ++i) {
                        const char c = p[i];
                        if (!std::isxdigit((unsigned char)c))
                            return false;
                        v = v * 16 + (unsigned)(std::isdigit((unsigned char)c) ? c - '0'
                                                                                : (std::tolower(c) - 'a' + 10));
                    }
                    if (v >= 0x80)
                        return false;  // device names and keys are ASCII
                    out += (char)v;
                    p += 4;
                    break;
                }
                default: return false;
                }
                ++p;
            } else {
                out += *p++;
            }
        }
        if (*p != '"')
            return false;
        ++p;
        return true;
    }
    bool value(JVal &v)
    {
        if (++depth > 32)
            return false;
        ws();
        bool ok = false;
        if (*p == '{') {
            ++p;
            v.kind = JVal::OBJ;
            ws();
            if (*p == '}') {
                ++p;
                ok = true;
            } else {
                for (;;) {
                    ws();
                    std::string key;
                    if (!string(key))
                        break;
                    ws();
                    if (*p != ':')
                        break;
                    ++p;
                    JVal child;
                    if (!value(child))
                        break;
                    v.obj.emplace_back(std::move(key), std::move(child));
                    ws();
                    if (*p == ',') {
                        ++p;
                        continue;
                    }
                    if (*p == '}') {
                        ++p;
                        ok = true;
                    }
                    break;
                }
            }
        } else if (*p == '[') {
            ++p;
            v.kind = JVal::ARR;
            ws();
            if (*p == ']') {
                ++p;
                ok = true;
            } else {
                for (;;) {
                    JVal child;
                    if (!value(child))
                        break;
                    v.arr.push_back(std::move(child));
                    ws();
                    if (*p == ',') {
                        ++p;
                        continue;
                    }
                    if (*p == ']') {
                        ++p;
                        ok = true;
                    }
                    break;
                }
            }
        } else if (*p == '"') {
            v.kind = JVal::STR;
            ok = string(v.str);
        } else if (lit("true")) {
            v.kind = JVal::BOOL;
            v.num = 1;
            ok = true;
        } else if (lit("false")) {
            v.kind = JVal::BOOL;
            ok = true;
        } else if (lit("null")) {
            ok = true;
        } else if (*p == '-' || std::isdigit((unsigned char)*p)) {
            char *end = nullptr;
            v.kind = JVal::NUM;
            v.num = std::strtod(p, &end);
            ok = end != p && std::isfinite(v.num);
            p = end;
        }
        --depth;
        return ok;
    }
};

inline bool json_parse(const char *text, JVal &out)
{
    JReader r{text};
    if (!r.value(out))
        return false;
    r.ws();
    return *r.p == '\0';
}

inline bool json_int(const JVal *v, int64_t lo, int64_t hi, int64_t *out)
{
    if (!v || v->kind != JVal::NUM || v->num != std::floor(v->num) || v->num < (double)lo ||
        v->num > (double)hi)
        return false;
    *out = (int64_t)v->num;
    return true;
}

// Entries of a tuning text written for this GPU (name and SM count must match); false
// when the text is malformed, of another format or from another GPU.
inline bool tuning_from_json(const char *text, const char *gpu, int sms,
                             std::map<TuneKey, std::vector<int>> *out)
{
    JVal root;
    if (!json_parse(text, root) || root.kind != JVal::OBJ)
        return false;
    int64_t fmt = 0, s = 0;
    const JVal *g = root.get("gpu");
    const JVal *ents = root.get("entries");
    if (!json_int(root.get("format"), 0, 1 << 20, &fmt) || fmt != kTuningFormat || !g ||
        g->kind != JVal::STR || g->str != gpu || !json_int(root.get("sms"), 1, 1 << 20, &s) ||
        s != sms || !ents || ents->kind != JVal::ARR)
        return false;
    std::map<TuneKey, std::vector<int>> res;
    for (const JVal &e : ents->arr) {
        if (e.kind != JVal::OBJ)
            return false;
        int64_t f[10];
        const char *names[10] = {"m", "n", "iters", "prec", "schedule", "norm", "polish",
                                 "mode", "hp_steps", "fuse"};
        const int64_t lo[10] = {1, 1, 0, 0, 0, 0, 0, 0, -1, 0};
        const int64_t hi[10] = {1 << 20, 1 << 20, 1000, 3, 2, 2, 1, 1, 1000, 1};
        for (int i = 0; i < 10; ++i)
            if (!json_int(e.get(names[i]), lo[i], hi[i], &f[i]))
                return false;
        const JVal *ell0 = e.get("ell0"), *delta = e.get("delta"), *w = e.get("widths");
        if (!ell0 || ell0->kind != JVal::NUM || !(ell0->num > 0.0 && ell0->num < 1.0) || !delta ||
            delta->kind != JVal::NUM || delta->num < 0.0 || !w || w->kind != JVal::ARR ||
            w->arr.empty())
            return false;
        std::vector<int> widths;
        for (const JVal &x : w->arr) {
            int64_t b = 0;
            if (!json_int(&x, 128, kBnPair, &b) || (b != 128 && b != 256 && b != kBnPair))
                return false;
            widths.push_back((int)b);
        }
        TuneKey k{f[0], f[1], (int)f[2], (int)f[3], (int)f[4], (int)f[5], (int)f[6], (int)f[7],
                  (int)f[8], ell0->num, delta->num, (int)f[9]};
        res[k] = std::move(widths);
    }
    *out = std::move(res);
    return true;
}

} // namespace svt
