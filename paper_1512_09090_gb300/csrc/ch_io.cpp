// CH file format, array views and the thread-local error message.
//
// File layout (little-endian): magic "ISOCH\0\0\2", then int32 n, int32 L,
// int32 max_w, int32 reserved, int64 m, int64 m_down, int64 m_up, int64
// shortcuts, then the arrays perm, bfs, level_off, down_off, down_src, down_w,
// up_off, up_dst, up_w, orig_off, orig_head, orig_id in that order.  Loading
// checks every size and id so a truncated or foreign file is rejected.
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>

#include "ch_internal.h"
#include "../../include/iso.h"

namespace iso {
static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }
}  // namespace iso

extern "C" const char* iso_last_error(void) { return iso::g_last_error.c_str(); }
extern "C" const char* iso_version(void) { return "iso-gb300 0.2 (sm_103a)"; }

namespace {
const char kMagic[8] = {'I', 'S', 'O', 'C', 'H', 0, 0, 2};

template <class T>
bool put(FILE* f, const std::vector<T>& v) {
    return v.empty() || std::fwrite(v.data(), sizeof(T), v.size(), f) == v.size();
}
template <class T>
bool get(FILE* f, std::vector<T>& v, size_t count) {
    try { v.resize(count); } catch (...) { return false; }
    return count == 0 || std::fread(v.data(), sizeof(T), count, f) == count;
}
}  // namespace

extern "C" int iso_ch_view_arrays(const iso_ch* ch, iso_ch_view* o) {
    iso::clear_error();
    if (!ch || !o) { iso::set_error("iso_ch_view_arrays: NULL argument"); return ISO_E_INVAL; }
    o->perm = ch->perm.data(); o->pos = ch->pos.data(); o->level_off = ch->level_off.data();
    o->down_off = ch->down_off.data(); o->down_src = ch->down_src.data(); o->down_w = ch->down_w.data();
    o->up_off = ch->up_off.data(); o->up_dst = ch->up_dst.data(); o->up_w = ch->up_w.data();
    o->orig_off = ch->orig_off.data(); o->orig_head = ch->orig_head.data(); o->orig_id = ch->orig_id.data();
    o->bfs = ch->bfs.data();
    return ISO_OK;
}

extern "C" int iso_save_ch(const iso_ch* ch, const char* path) {
    iso::clear_error();
    if (!ch || !path) { iso::set_error("iso_save_ch: NULL argument"); return ISO_E_INVAL; }
    FILE* f = std::fopen(path, "wb");
    if (!f) { iso::set_error("iso_save_ch: cannot open %s", path); return ISO_E_IO; }
    int32_t hdr32[4] = {ch->n, ch->L, ch->max_w, 0};
    int64_t hdr64[4] = {ch->m, ch->down_off.back(), ch->up_off.back(), ch->shortcuts};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr32, 4, 4, f) == 4 &&
              std::fwrite(hdr64, 8, 4, f) == 4 && put(f, ch->perm) && put(f, ch->bfs) && put(f, ch->level_off) &&
              put(f, ch->down_off) && put(f, ch->down_src) && put(f, ch->down_w) &&
              put(f, ch->up_off) && put(f, ch->up_dst) && put(f, ch->up_w) && put(f, ch->orig_off) &&
              put(f, ch->orig_head) && put(f, ch->orig_id);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) { iso::set_error("iso_save_ch: write to %s failed", path); return ISO_E_IO; }
    return ISO_OK;
}

static bool offsets_ok(const std::vector<int64_t>& off, int64_t total) {
    if (off.empty() || off[0] != 0 || off.back() != total) return false;
    for (size_t i = 1; i < off.size(); ++i)
        if (off[i] < off[i - 1]) return false;
    return true;
}

static bool ids_ok(const std::vector<int32_t>& ids, int32_t n) {
    for (int32_t x : ids)
        if (x < 0 || x >= n) return false;
    return true;
}

extern "C" int iso_load_ch(const char* path, iso_ch** out) {
    iso::clear_error();
    if (!path || !out) { iso::set_error("iso_load_ch: NULL argument"); return ISO_E_INVAL; }
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) { iso::set_error("iso_load_ch: cannot open %s", path); return ISO_E_IO; }
    std::unique_ptr<iso_ch> ch(new iso_ch());
    char magic[8];
    int32_t h32[4];
    int64_t h64[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(h32, 4, 4, f) == 4 && std::fread(h64, 8, 4, f) == 4;
    if (ok) {
        ch->n = h32[0]; ch->L = h32[1]; ch->max_w = h32[2];
        ch->m = h64[0]; ch->shortcuts = h64[3];
        int64_t md = h64[1], mu = h64[2];
        ok = ch->n > 0 && ch->L > 0 && ch->L <= ch->n && ch->m >= 0 && ch->m <= INT32_MAX && md >= 0 &&
             mu >= 0 && md <= (int64_t)UINT32_MAX && mu <= (int64_t)UINT32_MAX && ch->max_w >= 0 &&
             ch->max_w <= iso::kMaxWeight;
        size_t n = (size_t)ch->n;
        ok = ok && get(f, ch->perm, n) && get(f, ch->bfs, n) && get(f, ch->level_off, (size_t)ch->L + 1) &&
             get(f, ch->down_off, n + 1) && get(f, ch->down_src, (size_t)md) && get(f, ch->down_w, (size_t)md) &&
             get(f, ch->up_off, n + 1) && get(f, ch->up_dst, (size_t)mu) && get(f, ch->up_w, (size_t)mu) &&
             get(f, ch->orig_off, n + 1) && get(f, ch->orig_head, (size_t)ch->m) &&
             get(f, ch->orig_id, (size_t)ch->m);
        char extra;
        ok = ok && std::fread(&extra, 1, 1, f) == 0;
        ok = ok && offsets_ok(ch->down_off, md) && offsets_ok(ch->up_off, mu) && offsets_ok(ch->orig_off, ch->m) &&
             ids_ok(ch->perm, ch->n) && ids_ok(ch->bfs, ch->n) && ids_ok(ch->down_src, ch->n) && ids_ok(ch->up_dst, ch->n) &&
             ids_ok(ch->orig_head, ch->n) && ch->level_off[0] == 0 && ch->level_off[ch->L] == ch->n;
        if (ok) {
            ch->pos.assign(n, -1);
            for (int32_t p = 0; p < ch->n && ok; ++p) {
                if (ch->pos[ch->perm[p]] != -1) ok = false;
                else ch->pos[ch->perm[p]] = p;
            }
            for (int32_t j = 0; j < ch->L && ok; ++j) ok = ch->level_off[j] <= ch->level_off[j + 1];
            for (int32_t x : ch->orig_id) if (x < 0 || x >= ch->m) { ok = false; break; }
            for (int32_t x : ch->down_w) if (x < 0) { ok = false; break; }
            for (int32_t x : ch->up_w) if (x < 0) { ok = false; break; }
            // the BFS ranks are a permutation (emission lays tails out by them)
            std::vector<char> seen(n, 0);
            for (int32_t x : ch->bfs) {
                if (seen[(size_t)x]) { ok = false; break; }
                seen[(size_t)x] = 1;
            }
            // every downward arc comes from a higher level and every upward arc
            // goes to one: the sweep's order depends on it (level block 0 = top)
            std::vector<int32_t> block(n);
            for (int32_t j = 0; j < ch->L && ok; ++j)
                for (int32_t v = ch->level_off[j]; v < ch->level_off[j + 1]; ++v) block[(size_t)v] = j;
            for (size_t v = 0; v < n && ok; ++v) {
                for (int64_t a = ch->down_off[v]; a < ch->down_off[v + 1]; ++a)
                    if (block[(size_t)ch->down_src[(size_t)a]] >= block[v]) { ok = false; break; }
                for (int64_t a = ch->up_off[v]; a < ch->up_off[v + 1] && ok; ++a)
                    if (block[(size_t)ch->up_dst[(size_t)a]] >= block[v]) { ok = false; break; }
            }
        }
    }
    std::fclose(f);
    if (!ok) { iso::set_error("iso_load_ch: %s is not a valid CH file", path); return ISO_E_IO; }
    *out = ch.release();
    return ISO_OK;
}
