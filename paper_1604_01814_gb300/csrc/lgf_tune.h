// Text form of the autotuner's persisted choices (plain C++, no CUDA): the
// library and its host tests share it.
//
// One line per tuned item, "key -> value", where key and value are
// space-free tokens joined by single spaces; lines starting with '#' are
// comments.  A Poisson plan's key names everything its timing depends on
// (precision, block edge, block extents of source and target and their
// offset, field count) and its value the choice:
//   P f32 b16 s4,2,4 t67,4,4 o-1,-1,0 nf3 -> x1 y1 bx0 by0 bz0 z0
// A batch's key is a hash of its shape (block sets, operations, field
// counts) and its value the branch count:
//   B f32 9f3a... -> nb4
// Later lines win, so a file can be appended to as items are tuned.
#pragma once
#include <cstdio>
#include <map>
#include <sstream>
#include <string>

namespace lgf {

struct TuneChoiceText {
    int shift[2] = {0, 0};
    int bump[3] = {0, 0, 0};
    int zvar = 0;
    int fuse = 0;
};

inline std::string tune_plan_key(bool f64, int b, const int nbs[3], const int nbt[3], const int off[3], int nf)
{
    std::ostringstream o;
    o << "P " << (f64 ? "f64" : "f32") << " b" << b << " s" << nbs[0] << ',' << nbs[1] << ',' << nbs[2] << " t"
      << nbt[0] << ',' << nbt[1] << ',' << nbt[2] << " o" << off[0] << ',' << off[1] << ',' << off[2] << " nf" << nf;
    return o.str();
}

inline std::string tune_plan_value(const TuneChoiceText &c)
{
    std::ostringstream o;
    o << "x" << c.shift[0] << " y" << c.shift[1] << " bx" << c.bump[0] << " by" << c.bump[1] << " bz" << c.bump[2]
      << " z" << c.zvar << " f" << c.fuse;
    return o.str();
}

// Parse a plan value; false if malformed or out of range.
inline bool tune_parse_plan_value(const std::string &v, TuneChoiceText *c)
{
    TuneChoiceText t;
    // (files written before the fused inverse existed end after the z field:
    // the inverse then stays apart, the default)
    const int nread = std::sscanf(v.c_str(), "x%d y%d bx%d by%d bz%d z%d f%d", &t.shift[0], &t.shift[1], &t.bump[0],
                                  &t.bump[1], &t.bump[2], &t.zvar, &t.fuse);
    if (nread != 6 && nread != 7) return false;
    if (t.fuse < 0 || t.fuse > 1) return false;
    for (int d = 0; d < 2; ++d)
        if (t.shift[d] < 0 || t.shift[d] > 1) return false;
    for (int d = 0; d < 3; ++d)
        if (t.bump[d] < 0 || t.bump[d] > 2) return false;
    if (t.zvar < 0 || t.zvar > 1) return false;
    *c = t;
    return true;
}

inline std::string tune_batch_key(bool f64, unsigned long long hash)
{
    char buf[64];
    std::snprintf(buf, sizeof buf, "B %s %016llx", f64 ? "f64" : "f32", hash);
    return buf;
}

// 64-bit FNV-1a of a byte range (the batch shape).
inline unsigned long long tune_hash(const unsigned char *p, size_t n)
{
    unsigned long long h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Read "key -> value" lines into m (later lines win).  Returns the number of
// lines taken; malformed lines are skipped.
inline int tune_parse(const std::string &text, std::map<std::string, std::string> *m)
{
    std::istringstream in(text);
    std::string line;
    int n = 0;
    while (std::getline(in, line)) {
        if (line.empty() || line[0] == '#') continue;
        const size_t a = line.find(" -> ");
        if (a == std::string::npos || a == 0 || a + 4 >= line.size()) continue;
        (*m)[line.substr(0, a)] = line.substr(a + 4);
        ++n;
    }
    return n;
}

inline std::string tune_line(const std::string &key, const std::string &value) { return key + " -> " + value + "\n"; }

}  // namespace lgf
