// Argument-spec parser and statement analysis (see spec.h).
#include "spec.h"

#include <cctype>
#include <cstring>
#include <set>

namespace pyc {

namespace {

const std::set<std::string>& cxx_keywords() {
  static const std::set<std::string> k = {
      "alignas", "alignof", "and", "asm", "auto", "bool", "break", "case", "catch", "char",
      "class", "const", "constexpr", "const_cast", "continue", "decltype", "default",
      "delete", "do", "double", "dynamic_cast", "else", "enum", "explicit", "export",
      "extern", "false", "float", "for", "friend", "goto", "if", "inline", "int", "long",
      "mutable", "namespace", "new", "noexcept", "not", "nullptr", "operator", "or",
      "private", "protected", "public", "register", "reinterpret_cast", "return", "short",
      "signed", "sizeof", "static", "static_assert", "static_cast", "struct", "switch",
      "template", "this", "throw", "true", "try", "typedef", "typeid", "typename", "union",
      "unsigned", "using", "virtual", "void", "volatile", "while", "restrict",
      "__restrict__", "__restrict", "half", "bf16", "bfloat16"};
  return k;
}

bool is_ident_start(char c) { return std::isalpha((unsigned char)c) || c == '_'; }
bool is_ident_char(char c) { return std::isalnum((unsigned char)c) || c == '_'; }

bool valid_user_name(const std::string& n) {
  if (n.empty() || !is_ident_start(n[0])) return false;
  for (char c : n)
    if (!is_ident_char(c)) return false;
  if (n == "i" || n == "n") return false;
  if (n.rfind("pyc_", 0) == 0 || n.rfind("__", 0) == 0) return false;
  return cxx_keywords().count(n) == 0;
}

// Maps a sequence of type words to a dtype.
bool type_from_words(const std::vector<std::string>& w, pyc_dtype* out) {
  std::string s;
  for (size_t j = 0; j < w.size(); ++j) s += (j ? " " : "") + w[j];
  static const std::pair<const char*, pyc_dtype> table[] = {
      {"float", PYC_F32},
      {"double", PYC_F64},
      {"int", PYC_I32},
      {"signed", PYC_I32},
      {"signed int", PYC_I32},
      {"int32_t", PYC_I32},
      {"unsigned", PYC_U32},
      {"unsigned int", PYC_U32},
      {"uint32_t", PYC_U32},
      {"long long", PYC_I64},
      {"long long int", PYC_I64},
      {"signed long long", PYC_I64},
      {"long", PYC_I64},
      {"long int", PYC_I64},
      {"int64_t", PYC_I64},
      {"unsigned long long", PYC_U64},
      {"unsigned long long int", PYC_U64},
      {"unsigned long", PYC_U64},
      {"uint64_t", PYC_U64},
      {"size_t", PYC_U64},
      {"short", PYC_I16},
      {"short int", PYC_I16},
      {"int16_t", PYC_I16},
      {"unsigned short", PYC_U16},
      {"unsigned short int", PYC_U16},
      {"uint16_t", PYC_U16},
      {"signed char", PYC_I8},
      {"int8_t", PYC_I8},
      {"unsigned char", PYC_U8},
      {"uint8_t", PYC_U8},
      {"__nv_bfloat16", PYC_BF16},
      {"bfloat16", PYC_BF16},
      {"bf16", PYC_BF16},
      {"__half", PYC_F16},
      {"half", PYC_F16},
  };
  for (auto& e : table)
    if (s == e.first) {
      *out = e.second;
      return true;
    }
  return false;
}

const char* kPunct3[] = {"<<=", ">>=", "...", "->*"};
const char* kPunct2[] = {"->", "++", "--", "<<", ">>", "<=", ">=", "==", "!=", "&&",
                         "||", "+=", "-=", "*=", "/=", "%=", "&=", "|=", "^=", "::"};
const char* kPunct1 = "+-*/%<>=!&|^~?:;,.()[]{}";

bool is_assign_op(const std::string& t) {
  return t == "=" || t == "+=" || t == "-=" || t == "*=" || t == "/=" || t == "%=" ||
         t == "&=" || t == "|=" || t == "^=" || t == "<<=" || t == ">>=";
}

void check_balanced(const std::vector<Token>& t, const char* what) {
  std::string stack;
  for (auto& k : t) {
    if (k.kind != Token::Punct) continue;
    char c = k.text.size() == 1 ? k.text[0] : 0;
    if (c == '(' || c == '[' || c == '{') stack.push_back(c);
    if (c == ')' || c == ']' || c == '}') {
      char want = c == ')' ? '(' : c == ']' ? '[' : '{';
      if (stack.empty() || stack.back() != want)
        fail(PYC_E_PARSE, std::string(what) + ": unbalanced '" + k.text + "'");
      stack.pop_back();
    }
  }
  if (!stack.empty()) fail(PYC_E_PARSE, std::string(what) + ": unclosed '" + stack.back() + "'");
}

void check_forbidden(const std::vector<Token>& t, const char* what) {
  for (auto& k : t)
    if (k.kind == Token::Ident &&
        (k.text == "return" || k.text == "goto" || k.text == "asm" ||
         k.text == "__syncthreads" || k.text.rfind("pyc_", 0) == 0))
      fail(PYC_E_PARSE, std::string(what) + ": '" + k.text + "' is not allowed here");
}

}  // namespace

std::vector<Token> tokenize(const std::string& s) {
  std::vector<Token> out;
  size_t p = 0, n = s.size();
  while (p < n) {
    char c = s[p];
    if (std::isspace((unsigned char)c)) {
      ++p;
      continue;
    }
    if (c == '/' && p + 1 < n && s[p + 1] == '/') {
      while (p < n && s[p] != '\n') ++p;
      continue;
    }
    if (c == '/' && p + 1 < n && s[p + 1] == '*') {
      size_t e = s.find("*/", p + 2);
      if (e == std::string::npos) fail(PYC_E_PARSE, "unterminated comment");
      p = e + 2;
      continue;
    }
    if (c == '#') fail(PYC_E_PARSE, "preprocessor directives are not allowed in statements");
    if (is_ident_start(c)) {
      size_t q = p;
      while (q < n && is_ident_char(s[q])) ++q;
      out.push_back({Token::Ident, s.substr(p, q - p)});
      p = q;
      continue;
    }
    if (std::isdigit((unsigned char)c) || (c == '.' && p + 1 < n && std::isdigit((unsigned char)s[p + 1]))) {
      size_t q = p;
      while (q < n) {
        char d = s[q];
        if (is_ident_char(d) || d == '.') {
          ++q;
        } else if ((d == '+' || d == '-') && q > p &&
                   (s[q - 1] == 'e' || s[q - 1] == 'E' || s[q - 1] == 'p' || s[q - 1] == 'P') &&
                   !(s[p] == '0' && q > p + 1 && (s[p + 1] == 'x' || s[p + 1] == 'X') &&
                     (s[q - 1] == 'e' || s[q - 1] == 'E'))) {
          ++q;
        } else {
          break;
        }
      }
      out.push_back({Token::Number, s.substr(p, q - p)});
      p = q;
      continue;
    }
    if (c == '"' || c == '\'') {
      size_t q = p + 1;
      while (q < n && s[q] != c) {
        if (s[q] == '\\') ++q;
        if (s[q] == '\n') break;
        ++q;
      }
      if (q >= n || s[q] != c) fail(PYC_E_PARSE, "unterminated literal");
      out.push_back({Token::String, s.substr(p, q - p + 1)});
      p = q + 1;
      continue;
    }
    bool matched = false;
    for (const char* op : kPunct3)
      if (s.compare(p, 3, op) == 0) {
        out.push_back({Token::Punct, op});
        p += 3;
        matched = true;
        break;
      }
    if (matched) continue;
    for (const char* op : kPunct2)
      if (s.compare(p, 2, op) == 0) {
        out.push_back({Token::Punct, op});
        p += 2;
        matched = true;
        break;
      }
    if (matched) continue;
    if (std::strchr(kPunct1, c) && c != 0) {
      out.push_back({Token::Punct, std::string(1, c)});
      ++p;
      continue;
    }
    fail(PYC_E_PARSE, std::string("unexpected character '") + c + "' in code");
  }
  return out;
}

std::string join_tokens(const std::vector<Token>& t) {
  std::string s;
  for (size_t j = 0; j < t.size(); ++j) {
    if (j) s += ' ';
    s += t[j].text;
  }
  return s;
}

ArgSpec parse_argspec(const std::string& text) {
  ArgSpec spec;
  std::vector<Token> toks = tokenize(text);
  if (toks.empty()) fail(PYC_E_PARSE, "empty argument list");
  std::vector<std::vector<Token>> decls(1);
  for (auto& t : toks) {
    if (t.kind == Token::Punct && t.text == ",")
      decls.emplace_back();
    else
      decls.back().push_back(t);
  }
  std::set<std::string> seen;
  int scalar_off = 0, args_off = 0, args_align = 1;
  for (auto& d : decls) {
    if (d.empty()) fail(PYC_E_PARSE, "empty parameter in argument list");
    Param p;
    std::vector<std::string> words;
    int stars = 0;
    for (size_t j = 0; j + 1 < d.size(); ++j) {
      const Token& t = d[j];
      if (t.kind == Token::Punct && t.text == "*") {
        ++stars;
      } else if (t.kind == Token::Ident) {
        if (t.text == "const") {
          p.is_const = true;
        } else if (t.text == "volatile" || t.text == "__restrict__" || t.text == "restrict" ||
                   t.text == "__restrict") {
          // qualifiers carry no meaning for the generated code
        } else {
          if (stars) fail(PYC_E_PARSE, "unexpected '" + t.text + "' after '*'");
          words.push_back(t.text);
        }
      } else {
        fail(PYC_E_PARSE, "unexpected '" + t.text + "' in parameter declaration");
      }
    }
    const Token& last = d.back();
    if (last.kind != Token::Ident) fail(PYC_E_PARSE, "parameter name missing");
    p.name = last.text;
    if (words.empty()) fail(PYC_E_PARSE, "type missing for '" + p.name + "'");
    if (words.size() == 1 && words[0] == "char")
      fail(PYC_E_PARSE, "plain 'char' has platform-dependent signedness; use signed char or unsigned char");
    if (!type_from_words(words, &p.dtype)) {
      std::string w;
      for (auto& x : words) w += x + " ";
      fail(PYC_E_PARSE, "unsupported type '" + w.substr(0, w.size() - 1) + "'");
    }
    if (stars > 1) fail(PYC_E_PARSE, "pointer-to-pointer parameter '" + p.name + "'");
    p.is_ptr = stars == 1;
    if (!valid_user_name(p.name))
      fail(PYC_E_PARSE, "invalid or reserved parameter name '" + p.name + "'");
    if (!seen.insert(p.name).second) fail(PYC_E_PARSE, "duplicate parameter '" + p.name + "'");
    int sz = p.is_ptr ? 8 : type_info(p.dtype).bytes;
    if (p.is_ptr) {
      p.ptr_slot = spec.num_ptrs++;
    } else {
      int tb = type_info(p.dtype).bytes;
      scalar_off = (scalar_off + tb - 1) / tb * tb;
      p.scalar_offset = scalar_off;
      scalar_off += tb;
    }
    args_off = (args_off + sz - 1) / sz * sz;
    p.args_offset = args_off;
    args_off += sz;
    if (sz > args_align) args_align = sz;
    spec.canonical += (spec.canonical.empty() ? "" : ", ") +
                      std::string(type_info(p.dtype).device_name) + (p.is_ptr ? " *" : " ") + p.name;
    spec.params.push_back(p);
  }
  int max_al = 1;
  for (auto& p : spec.params)
    if (!p.is_ptr) max_al = std::max(max_al, type_info(p.dtype).bytes);
  spec.scalar_bytes = (scalar_off + max_al - 1) / max_al * max_al;
  spec.args_align = args_align;
  spec.args_bytes = (args_off + args_align - 1) / args_align * args_align;
  return spec;
}

namespace {

bool is_member_at(const std::vector<Token>& t, size_t j) {
  return j > 0 && t[j - 1].kind == Token::Punct &&
         (t[j - 1].text == "." || t[j - 1].text == "->" || t[j - 1].text == "::");
}

bool is_index_i_at(const std::vector<Token>& t, size_t j) {
  return j + 3 < t.size() && t[j + 1].text == "[" && t[j + 2].text == "i" &&
         t[j + 2].kind == Token::Ident && t[j + 3].text == "]";
}

Param* find_array(ArgSpec& spec, const std::string& name) {
  for (auto& p : spec.params)
    if (p.is_ptr && p.name == name) return &p;
  return nullptr;
}

}  // namespace

void analyze_code(ArgSpec& spec, const std::string& code, bool expression) {
  const char* what = expression ? "map expression" : "statement";
  std::vector<Token> t = tokenize(code);
  check_balanced(t, what);
  check_forbidden(t, what);
  int depth = 0;
  for (size_t j = 0; j < t.size(); ++j) {
    const Token& k = t[j];
    if (k.kind == Token::Punct && (k.text == "(" || k.text == "[" || k.text == "{")) ++depth;
    if (k.kind == Token::Punct && (k.text == ")" || k.text == "]" || k.text == "}")) --depth;
    if (k.kind != Token::Ident || is_member_at(t, j)) continue;
    Param* p = find_array(spec, k.text);
    if (!p) continue;
    p->used = true;
    if (!is_index_i_at(t, j)) {
      p->raw = true;
      p->read = true;
      if (!expression) p->written = true;  // unknown use: assume both
      continue;
    }
    // address-of: '&' in unary position before name[i]
    if (j > 0 && t[j - 1].text == "&") {
      // a binary '&' follows an operand; anything else makes it address-of
      bool unary = true;
      if (j >= 2) {
        const Token& pp = t[j - 2];
        bool operand = pp.kind == Token::Ident || pp.kind == Token::Number ||
                       pp.kind == Token::String || pp.text == ")" || pp.text == "]";
        unary = !operand;
      }
      if (unary) {
        p->raw = true;
        p->read = true;
        if (!expression) p->written = true;
        continue;
      }
    }
    const std::string next = j + 4 < t.size() ? t[j + 4].text : "";
    const std::string prev = j > 0 ? t[j - 1].text : "";
    bool incdec = next == "++" || next == "--" || prev == "++" || prev == "--";
    if (is_assign_op(next) || incdec) {
      if (expression) {
        p->raw = true;  // side effects in a map expression: leave it to the compiler
        p->read = p->written = true;
        continue;
      }
      p->written = true;
      if (next != "=" || incdec) p->read = true;
      // a plain assignment that starts a top-level statement writes every element
      bool top = depth == 0 && next == "=" && !incdec &&
                 (j == 0 || t[j - 1].text == ";" || t[j - 1].text == "}");
      if (top) p->fully_written = true;
    } else {
      p->read = true;
    }
  }
  for (auto& p : spec.params) {
    if (!p.is_ptr || !p.used) continue;
    p.lifted = !p.raw;
    // an element the code may leave unwritten must be stored back unchanged
    if (p.lifted && p.written && !p.fully_written) p.read = true;
  }
}

std::string rewrite_lifted(ArgSpec& spec, const std::string& code) {
  std::vector<Token> t = tokenize(code);
  std::vector<Token> o;
  for (size_t j = 0; j < t.size(); ++j) {
    const Token& k = t[j];
    if (k.kind == Token::Ident && !is_member_at(t, j)) {
      Param* p = find_array(spec, k.text);
      if (p && p->lifted && is_index_i_at(t, j)) {
        o.push_back({Token::Ident, "pyc_r_" + p->name});
        o.push_back({Token::Punct, "["});
        o.push_back({Token::Ident, "pyc_k"});
        o.push_back({Token::Punct, "]"});
        j += 3;
        continue;
      }
    }
    o.push_back(k);
  }
  return join_tokens(o);
}

std::string analyze_and_rewrite(ArgSpec& spec, const std::string& code, bool expression) {
  analyze_code(spec, code, expression);
  return rewrite_lifted(spec, code);
}

std::string check_expression(const std::string& code, const char* what) {
  std::vector<Token> t = tokenize(code);
  if (t.empty()) fail(PYC_E_PARSE, std::string(what) + " is empty");
  check_balanced(t, what);
  check_forbidden(t, what);
  for (auto& k : t)
    if (k.kind == Token::Punct && (k.text == ";" || k.text == "{" || k.text == "}"))
      fail(PYC_E_PARSE, std::string(what) + " must be a single expression");
  return join_tokens(t);
}

}  // namespace pyc
