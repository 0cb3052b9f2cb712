// The batch autotuner's JSON store (see rr_tune_cache.h).  A small reader for
// the subset of JSON the file uses (objects, strings, numbers, true, false,
// null, arrays skipped) and a writer that replaces the file atomically.
#include "rr_tune_cache.h"

#include <unistd.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>

namespace rr {

namespace {

constexpr const char *kFormat = "rr-batch-tune-cache";
constexpr int kVersion = 1;

struct Reader {
    const std::string &s;
    size_t i = 0;
    bool ok = true;

    explicit Reader(const std::string &text) : s(text) {}

    void ws() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool string(std::string *out) {
        ws();
        if (i >= s.size() || s[i] != '"') return ok = false;
        ++i;
        out->clear();
        while (i < s.size() && s[i] != '"') {
            char c = s[i++];
            if (c == '\\') {
                if (i >= s.size()) return ok = false;
                const char e = s[i++];
                switch (e) {
                    case '"': c = '"'; break;
                    case '\\': c = '\\'; break;
                    case '/': c = '/'; break;
                    case 'b': c = '\b'; break;
                    case 'f': c = '\f'; break;
                    case 'n': c = '\n'; break;
                    case 'r': c = '\r'; break;
                    case 't': c = '\t'; break;
                    case 'u': {
                        if (i + 4 > s.size()) return ok = false;
                        const long v = std::strtol(s.substr(i, 4).c_str(), nullptr, 16);
                        i += 4;
                        c = v < 0x80 ? (char)v : '?';
                        break;
                    }
                    default: return ok = false;
                }
            }
            out->push_back(c);
        }
        if (i >= s.size()) return ok = false;
        ++i;
        return true;
    }
    bool number(double *out) {
        ws();
        const char *b = s.c_str() + i;
        char *e = nullptr;
        const double v = std::strtod(b, &e);
        if (e == b) return ok = false;
        i += (size_t)(e - b);
        *out = v;
        return true;
    }
    // Skips one value of any kind.
    bool skip() {
        ws();
        if (i >= s.size()) return ok = false;
        const char c = s[i];
        if (c == '"') {
            std::string t;
            return string(&t);
        }
        if (c == '{' || c == '[') {
            const char close = c == '{' ? '}' : ']';
            ++i;
            if (eat(close)) return true;
            do {
                if (c == '{') {
                    std::string k;
                    if (!string(&k) || !eat(':')) return ok = false;
                }
                if (!skip()) return false;
            } while (eat(','));
            return eat(close) || (ok = false);
        }
        for (const char *lit : {"true", "false", "null"}) {
            const size_t n = std::char_traits<char>::length(lit);
            if (s.compare(i, n, lit) == 0) {
                i += n;
                return true;
            }
        }
        double d;
        return number(&d);
    }
};

bool read_entry(Reader &r, TuneEntry *e) {
    if (!r.eat('{')) return false;
    if (r.eat('}')) return true;
    do {
        std::string k;
        if (!r.string(&k) || !r.eat(':')) return false;
        double v = 0.0;
        if (k == "key_bits" || k == "radix_bits" || k == "trace_block" || k == "layout" || k == "ms") {
            if (!r.number(&v) || !std::isfinite(v)) return false;
            if (k == "key_bits") e->key_bits = (uint32_t)v;
            if (k == "radix_bits") e->radix_bits = (uint32_t)v;
            if (k == "trace_block") e->trace_block = (uint32_t)v;
            if (k == "layout") e->layout = (int32_t)v;
            if (k == "ms") e->ms = v;
        } else if (!r.skip()) {
            return false;
        }
    } while (r.eat(','));
    return r.eat('}');
}

// Every entry of the file; false when the file is missing or malformed.
bool read_file(const std::string &path, std::map<std::string, TuneEntry> *out) {
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    Reader r(text);
    std::map<std::string, TuneEntry> m;
    bool format_ok = false, version_ok = false;
    if (!r.eat('{')) return false;
    if (!r.eat('}')) {
        do {
            std::string k;
            if (!r.string(&k) || !r.eat(':')) return false;
            if (k == "format") {
                std::string v;
                if (!r.string(&v)) return false;
                format_ok = v == kFormat;
            } else if (k == "version") {
                double v;
                if (!r.number(&v)) return false;
                version_ok = v == kVersion;
            } else if (k == "entries") {
                if (!r.eat('{')) return false;
                if (!r.eat('}')) {
                    do {
                        std::string key;
                        TuneEntry e;
                        if (!r.string(&key) || !r.eat(':') || !read_entry(r, &e)) return false;
                        m[key] = e;
                    } while (r.eat(','));
                    if (!r.eat('}')) return false;
                }
            } else if (!r.skip()) {
                return false;
            }
        } while (r.eat(','));
        if (!r.eat('}')) return false;
    }
    r.ws();
    if (!r.ok || r.i != text.size() || !format_ok || !version_ok) return false;
    *out = std::move(m);
    return true;
}

std::string quoted(const std::string &s) {
    std::string o = "\"";
    for (const char c : s) {
        if (c == '"' || c == '\\') {
            o.push_back('\\');
            o.push_back(c);
        } else if ((unsigned char)c < 0x20) {
            char b[8];
            std::snprintf(b, sizeof(b), "\\u%04x", (unsigned)(unsigned char)c);
            o += b;
        } else {
            o.push_back(c);
        }
    }
    return o + "\"";
}

}  // namespace

bool tune_cache_lookup(const std::string &path, const std::string &key, TuneEntry *e) {
    std::map<std::string, TuneEntry> m;
    if (!read_file(path, &m)) return false;
    const auto it = m.find(key);
    if (it == m.end()) return false;
    *e = it->second;
    return true;
}

bool tune_cache_store(const std::string &path, const std::string &key, const TuneEntry &e, std::string *err) {
    std::map<std::string, TuneEntry> m;
    read_file(path, &m);  // a missing or malformed file starts empty
    m[key] = e;
    std::ostringstream o;
    o << "{\"format\": " << quoted(kFormat) << ", \"version\": " << kVersion << ", \"entries\": {";
    bool first = true;
    for (const auto &kv : m) {
        char num[64];
        std::snprintf(num, sizeof(num), "%.6g", kv.second.ms);
        o << (first ? "\n  " : ",\n  ") << quoted(kv.first) << ": {\"key_bits\": " << kv.second.key_bits
          << ", \"radix_bits\": " << kv.second.radix_bits << ", \"trace_block\": " << kv.second.trace_block
          << ", \"layout\": " << kv.second.layout << ", \"ms\": " << num << "}";
        first = false;
    }
    o << "\n}}\n";
    // a name of its own per process and call, so that concurrent writers
    // never share a temporary file
    static std::atomic<uint64_t> serial{0};
    const std::string tmp = path + ".tmp." + std::to_string((long)getpid()) + "." + std::to_string(serial++);
    {
        std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
        if (!f) {
            *err = "cannot write " + tmp;
            return false;
        }
        f << o.str();
        f.flush();
        if (!f) {
            *err = "cannot write " + tmp;
            std::remove(tmp.c_str());
            return false;
        }
    }
    if (std::rename(tmp.c_str(), path.c_str()) != 0) {
        *err = "cannot rename " + tmp + " to " + path;
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace rr
