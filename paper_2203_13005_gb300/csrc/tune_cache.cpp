// The autotuner's cache of measured pipeline coefficients (Section III-A:
// Lemma 1's k1, k2, k3, a and the block size the local sweep chose), kept in
// a JSON file so that a later run on the same graph shape and GPU skips the
// measurements. The file is one JSON object whose members are
//   "<key>": {"k1": ..., "k2": ..., "k3": ..., "a": ..., "model_block_edges": ...,
//             "block_edges": ..., "sweep_best_ms": ...}
// written one member per line; the reader accepts exactly what the writer
// produces (members it cannot read are kept as they are).
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "engine.hpp"

namespace gxp {
namespace {

const char* kFields[] = {"k1", "k2", "k3", "a", "model_block_edges", "block_edges", "sweep_best_ms"};

double* field_of(gxp_tune_record& r, int i) {
    switch (i) {
        case 0: return &r.k1;
        case 1: return &r.k2;
        case 2: return &r.k3;
        case 3: return &r.a;
        case 4: return &r.model_block_edges;
        case 5: return &r.block_edges;
        default: return &r.sweep_best_ms;
    }
}

std::string clean_key(const char* key) {
    std::string k;
    for (const char* p = key; *p; ++p) k += (*p == '"' || *p == '\\' || *p == '\n') ? '_' : *p;
    return k;
}

// the file's members as (key, the rest of the line) pairs
std::vector<std::pair<std::string, std::string>> read_members(const char* path) {
    std::vector<std::pair<std::string, std::string>> out;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t q0 = line.find('"');
        if (q0 == std::string::npos) continue;
        const size_t q1 = line.find('"', q0 + 1);
        const size_t brace = line.find('{', q1 == std::string::npos ? 0 : q1);
        if (q1 == std::string::npos || brace == std::string::npos) continue;
        std::string body = line.substr(brace);
        while (!body.empty() && (body.back() == ',' || body.back() == ' ' || body.back() == '\r')) body.pop_back();
        out.emplace_back(line.substr(q0 + 1, q1 - q0 - 1), body);
    }
    return out;
}

bool parse_record(const std::string& body, gxp_tune_record* r) {
    gxp_tune_record x{};
    for (int i = 0; i < 7; ++i) {
        const std::string tag = std::string("\"") + kFields[i] + "\":";
        const size_t at = body.find(tag);
        if (at == std::string::npos) return false;
        const char* s = body.c_str() + at + tag.size();
        char* end = nullptr;
        errno = 0;
        const double v = std::strtod(s, &end);
        if (end == s || errno) return false;
        *field_of(x, i) = v;
    }
    *r = x;
    return true;
}

std::string format_record(const gxp_tune_record& r) {
    std::ostringstream o;
    o.precision(17);
    o << "{";
    gxp_tune_record x = r;
    for (int i = 0; i < 7; ++i) o << (i ? ", " : "") << "\"" << kFields[i] << "\": " << *field_of(x, i);
    o << "}";
    return o.str();
}

}  // namespace

bool tune_cache_get(const char* path, const char* key, gxp_tune_record* out) {
    const std::string k = clean_key(key);
    for (const auto& m : read_members(path))
        if (m.first == k) return parse_record(m.second, out);
    return false;
}

bool tune_cache_put(const char* path, const char* key, const gxp_tune_record& rec) {
    auto members = read_members(path);
    const std::string k = clean_key(key), body = format_record(rec);
    bool found = false;
    for (auto& m : members)
        if (m.first == k) {
            m.second = body;
            found = true;
        }
    if (!found) members.emplace_back(k, body);
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return false;
        f << "{\n";
        for (size_t i = 0; i < members.size(); ++i)
            f << "\"" << members[i].first << "\": " << members[i].second << (i + 1 < members.size() ? ",\n" : "\n");
        f << "}\n";
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace gxp
