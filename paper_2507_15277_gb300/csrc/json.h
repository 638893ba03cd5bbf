// Minimal JSON reader/writer helpers for manifests (objects, arrays, strings,
// numbers, true/false/null).  Enough for the files this library writes.
#pragma once

#include <cctype>
#include <cstdlib>
#include <map>
#include <memory>
#include <string>
#include <vector>

namespace pt {
namespace json {

struct Value {
    enum Kind { Null, Bool, Number, String, Array, Object } kind = Null;
    bool b = false;
    double num = 0;
    std::string str;
    std::vector<Value> arr;
    std::map<std::string, Value> obj;

    const Value *get(const std::string &k) const {
        if (kind != Object) return nullptr;
        auto it = obj.find(k);
        return it == obj.end() ? nullptr : &it->second;
    }
};

class Parser {
  public:
    explicit Parser(const std::string &s) : s_(s) {}
    bool parse(Value *out) {
        if (!value(out)) return false;
        ws();
        return i_ == s_.size();
    }

  private:
    const std::string &s_;
    size_t i_ = 0;
    int depth_ = 0;

    void ws() {
        while (i_ < s_.size() && std::isspace((unsigned char)s_[i_])) ++i_;
    }
    bool lit(const char *w) {
        size_t n = 0;
        while (w[n]) ++n;
        if (s_.compare(i_, n, w) != 0) return false;
        i_ += n;
        return true;
    }
    bool string(std::string *out) {
        if (i_ >= s_.size() || s_[i_] != '"') return false;
        ++i_;
        out->clear();
        while (i_ < s_.size() && s_[i_] != '"') {
            char c = s_[i_++];
            if (c == '\\') {
                if (i_ >= s_.size()) return false;
                char e = s_[i_++];
                switch (e) {
                    case '"': case '\\': case '/': out->push_back(e); break;
                    case 'n': out->push_back('\n'); break;
                    case 't': out->push_back('\t'); break;
                    case 'r': out->push_back('\r'); break;
                    case 'b': out->push_back('\b'); break;
                    case 'f': out->push_back('\f'); break;
                    default: return false;  // \u escapes are not produced by this library
                }
            } else {
                out->push_back(c);
            }
        }
        if (i_ >= s_.size()) return false;
        ++i_;
        return true;
    }
    bool value(Value *v) {
        if (++depth_ > 64) return false;
        ws();
        if (i_ >= s_.size()) return false;
        const char c = s_[i_];
        bool ok = false;
        if (c == '{') {
            v->kind = Value::Object;
            ++i_;
            ws();
            if (i_ < s_.size() && s_[i_] == '}') {
                ++i_;
                ok = true;
            } else {
                while (true) {
                    ws();
                    std::string key;
                    if (!string(&key)) break;
                    ws();
                    if (i_ >= s_.size() || s_[i_] != ':') break;
                    ++i_;
                    Value item;
                    if (!value(&item)) break;
                    v->obj[key] = std::move(item);
                    ws();
                    if (i_ < s_.size() && s_[i_] == ',') { ++i_; continue; }
                    if (i_ < s_.size() && s_[i_] == '}') { ++i_; ok = true; }
                    break;
                }
            }
        } else if (c == '[') {
            v->kind = Value::Array;
            ++i_;
            ws();
            if (i_ < s_.size() && s_[i_] == ']') {
                ++i_;
                ok = true;
            } else {
                while (true) {
                    Value item;
                    if (!value(&item)) break;
                    v->arr.push_back(std::move(item));
                    ws();
                    if (i_ < s_.size() && s_[i_] == ',') { ++i_; continue; }
                    if (i_ < s_.size() && s_[i_] == ']') { ++i_; ok = true; }
                    break;
                }
            }
        } else if (c == '"') {
            v->kind = Value::String;
            ok = string(&v->str);
        } else if (lit("true")) {
            v->kind = Value::Bool; v->b = true; ok = true;
        } else if (lit("false")) {
            v->kind = Value::Bool; v->b = false; ok = true;
        } else if (lit("null")) {
            v->kind = Value::Null; ok = true;
        } else {
            const char *start = s_.c_str() + i_;
            char *end = nullptr;
            v->num = std::strtod(start, &end);
            if (end != start) {
                v->kind = Value::Number;
                i_ += (size_t)(end - start);
                ok = true;
            }
        }
        --depth_;
        return ok;
    }
};

inline std::string quote(const std::string &s) {
    std::string o = "\"";
    for (char c : s) {
        if (c == '"' || c == '\\') { o.push_back('\\'); o.push_back(c); }
        else if (c == '\n') o += "\\n";
        else o.push_back(c);
    }
    o.push_back('"');
    return o;
}

}  // namespace json
}  // namespace pt
