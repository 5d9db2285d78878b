// Launch-shape tuning (host only): the defaults, range checks, and the
// autotuner cache's reader and selection (leiden_tuning_lookup). The cache is
// a small JSON file; the reader below accepts the JSON grammar (objects,
// arrays, strings with escapes, numbers, true/false/null) and keeps what the
// selection needs.
#include <cctype>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "engine.h"

namespace lgb {
namespace {

struct JValue {
    enum Kind { Null, Bool, Num, Str, Arr, Obj } kind = Null;
    double num = 0;
    std::string str;
    std::vector<JValue> arr;
    std::vector<std::pair<std::string, JValue>> obj;
    const JValue *get(const std::string &k) const {
        for (auto &kv : obj)
            if (kv.first == k) return &kv.second;
        return nullptr;
    }
};

struct JParser {
    const std::string &t;
    size_t i = 0;
    bool ok = true;
    explicit JParser(const std::string &text) : t(text) {}
    void ws() {
        while (i < t.size() && std::isspace((unsigned char)t[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < t.size() && t[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    std::string string() {
        std::string out;
        if (!eat('"')) {
            ok = false;
            return out;
        }
        while (i < t.size() && t[i] != '"') {
            char c = t[i++];
            if (c == '\\' && i < t.size()) {
                const char e = t[i++];
                switch (e) {
                    case 'n': c = '\n'; break;
                    case 't': c = '\t'; break;
                    case 'r': c = '\r'; break;
                    case 'b': c = '\b'; break;
                    case 'f': c = '\f'; break;
                    case 'u':  // code points are kept as '?' (names here are ASCII)
                        i += 4;
                        c = '?';
                        break;
                    default: c = e;
                }
            }
            out.push_back(c);
        }
        if (i >= t.size()) ok = false;
        ++i;
        return out;
    }
    JValue value(int depth = 0) {
        JValue v;
        ws();
        if (depth > 64 || i >= t.size()) {
            ok = false;
            return v;
        }
        const char c = t[i];
        if (c == '{') {
            ++i;
            v.kind = JValue::Obj;
            if (eat('}')) return v;
            do {
                std::string k = string();
                if (!ok || !eat(':')) {
                    ok = false;
                    return v;
                }
                v.obj.emplace_back(k, value(depth + 1));
            } while (ok && eat(','));
            if (!eat('}')) ok = false;
        } else if (c == '[') {
            ++i;
            v.kind = JValue::Arr;
            if (eat(']')) return v;
            do v.arr.push_back(value(depth + 1));
            while (ok && eat(','));
            if (!eat(']')) ok = false;
        } else if (c == '"') {
            v.kind = JValue::Str;
            v.str = string();
        } else if (t.compare(i, 4, "true") == 0) {
            v.kind = JValue::Bool;
            v.num = 1;
            i += 4;
        } else if (t.compare(i, 5, "false") == 0) {
            v.kind = JValue::Bool;
            i += 5;
        } else if (t.compare(i, 4, "null") == 0) {
            i += 4;
        } else {
            char *end = nullptr;
            v.num = std::strtod(t.c_str() + i, &end);
            if (end == t.c_str() + i) ok = false;
            else i = (size_t)(end - t.c_str());
            v.kind = JValue::Num;
        }
        return v;
    }
};

bool read_file(const char *path, std::string &out) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    char buf[65536];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, k);
    std::fclose(f);
    return true;
}

}  // namespace

// The defaults: the largest bins the kernels' registers and shared-memory
// tables hold, as many persistent blocks as fit, and 2048 vertices per block
// below a full grid (a step's latency grows with the vertices each thread
// takes in turn; 4096 measured slower than 2048 on the aggregated passes of
// the road workload).
void tuning_default(leiden_tuning &t) {
    t = leiden_tuning{};
    t.thread_max_deg = 8;
    t.warp_max_deg = 256;
    t.block_max_deg = 2048;
    t.coop_blocks_per_sm = 0;
    t.vertices_per_block = 2048;
    t.list_order_min_vertices = 1 << 20;
}

bool tuning_valid(const leiden_tuning &t) {
    return t.thread_max_deg >= 1 && t.thread_max_deg <= 8 && t.warp_max_deg >= 32 && t.warp_max_deg <= 256 &&
           t.block_max_deg >= 128 && t.block_max_deg <= 2048 && t.block_max_deg >= t.warp_max_deg &&
           t.coop_blocks_per_sm >= 0 && t.coop_blocks_per_sm <= 32 && t.vertices_per_block >= 256 &&
           t.vertices_per_block <= 65536 && t.list_order_min_vertices >= 0;
}

leiden_status tuning_lookup(const char *path, const char *gpu, int64_t n, int64_t nnz, int64_t maxdeg,
                            leiden_tuning &out) {
    std::string text;
    if (!path || !gpu || !read_file(path, text)) {
        set_last_error(std::string("tuning cache cannot be read: ") + (path ? path : "(null)"));
        return LEIDEN_ERR_INVALID;
    }
    JParser ps(text);
    const JValue root = ps.value();
    const JValue *entries = root.kind == JValue::Obj ? root.get("entries") : nullptr;
    if (!ps.ok || !entries || entries->kind != JValue::Arr) {
        set_last_error("tuning cache is not a JSON object with an \"entries\" array");
        return LEIDEN_ERR_INVALID;
    }
    const int heavy = (double)maxdeg * (double)n > 64.0 * (double)nnz ? 1 : 0;
    const int ln = n > 0 ? (int)std::lround(std::log2((double)n)) : 0;
    const int lm = (n > 0 && nnz > 0) ? (int)std::lround(std::log2((double)nnz / (double)n)) : 0;
    const JValue *best = nullptr;
    double best_d = 0;
    for (const JValue &e : entries->arr) {
        if (e.kind != JValue::Obj) continue;
        const JValue *g = e.get("gpu"), *h = e.get("heavy_tailed"), *a = e.get("log2_vertices"),
                     *b = e.get("log2_mean_degree");
        if (!g || g->kind != JValue::Str || g->str != gpu || !h || !a || !b) continue;
        if ((int)h->num != heavy) continue;
        const double d = std::fabs(a->num - ln) + std::fabs(b->num - lm);
        if (!best || d < best_d) {
            best = &e;
            best_d = d;
        }
    }
    if (!best) {
        set_last_error("no tuning cache entry for this GPU and graph class");
        return LEIDEN_ERR_INVALID;
    }
    leiden_tuning t;
    tuning_default(t);
    auto take = [&](const char *k, int32_t &dst) {
        const JValue *v = best->get(k);
        if (v && v->kind == JValue::Num) dst = (int32_t)v->num;
    };
    take("thread_max_deg", t.thread_max_deg);
    take("warp_max_deg", t.warp_max_deg);
    take("block_max_deg", t.block_max_deg);
    take("coop_blocks_per_sm", t.coop_blocks_per_sm);
    take("vertices_per_block", t.vertices_per_block);
    take("list_order_min_vertices", t.list_order_min_vertices);
    if (!tuning_valid(t)) {
        set_last_error("tuning cache entry outside the valid ranges");
        return LEIDEN_ERR_INVALID;
    }
    out = t;
    return LEIDEN_OK;
}

}  // namespace lgb
