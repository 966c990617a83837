// Fused array expressions (Sec. 3.2.3-3.2.4): a nested arithmetic expression over
// equal-length arrays and scalars becomes ONE map (or map-reduce) kernel instead of
// one kernel and one temporary array per operation.  See include/pyc.h for the
// prefix syntax; this file parses it, types every node with C-style promotion
// (weak literals), and emits a fully parenthesised C expression with explicit
// conversions, which the map / map-reduce generators then compile.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "handles.h"

namespace pyc {

namespace {

// Value types of expression nodes, in promotion order.
enum class VT { I32 = 0, I64 = 1, F32 = 2, F64 = 3 };

const char* vt_name(VT t) {
  switch (t) {
    case VT::I32: return "int";
    case VT::I64: return "long long";
    case VT::F32: return "float";
    default: return "double";
  }
}
bool vt_float(VT t) { return t == VT::F32 || t == VT::F64; }

struct Node {
  std::string op;  // "$" array leaf, "%" scalar leaf, "#" literal, else an operator
  int slot = -1;
  std::string literal;
  bool lit_float = false;
  std::vector<std::unique_ptr<Node>> kids;
  VT type = VT::I32;
  bool weak = false;  // a literal: takes the other operand's type
};

struct Arg {
  pyc_dtype dtype;
  bool is_array;
};

struct Parser {
  const std::string& s;
  size_t p = 0;
  explicit Parser(const std::string& text) : s(text) {}

  [[noreturn]] void error(const std::string& m) {
    fail(PYC_E_PARSE, "expression: " + m + " at offset " + std::to_string(p) + " in '" + s + "'");
  }
  void skip() {
    while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
  }
  std::string token() {
    skip();
    size_t b = p;
    while (p < s.size() && !std::isspace((unsigned char)s[p]) && s[p] != '(' && s[p] != ')') ++p;
    if (b == p) error("expected a token");
    return s.substr(b, p - b);
  }
  std::unique_ptr<Node> parse() {
    skip();
    if (p >= s.size()) error("unexpected end");
    auto n = std::make_unique<Node>();
    if (s[p] == '(') {
      ++p;
      n->op = token();
      for (;;) {
        skip();
        if (p >= s.size()) error("missing ')'");
        if (s[p] == ')') {
          ++p;
          break;
        }
        n->kids.push_back(parse());
      }
      return n;
    }
    if (s[p] == ')') error("unexpected ')'");
    std::string t = token();
    if (t[0] == '$' || t[0] == '%') {
      n->op = t.substr(0, 1);
      char* end = nullptr;
      long k = std::strtol(t.c_str() + 1, &end, 10);
      if (t.size() < 2 || *end || k < 0 || k > 4096) error("bad argument reference '" + t + "'");
      n->slot = (int)k;
      return n;
    }
    // numeric literal: digits, optional fraction / exponent; no suffixes
    char* end = nullptr;
    std::strtod(t.c_str(), &end);
    if (*end || t.find_first_not_of("0123456789.eE+-") != std::string::npos)
      error("bad literal '" + t + "'");
    n->op = "#";
    n->literal = t;
    n->lit_float = t.find_first_of(".eE") != std::string::npos;
    return n;
  }
};

const char* const kUnary[] = {"neg", "abs", "exp", "exp2", "log", "log2", "sin", "cos", "tan",
                              "tanh", "sqrt", "rsqrt", "floor", "ceil"};
const char* const kBinary[] = {"+", "-", "*", "/", "min", "max", "pow",
                               "<", "<=", ">", ">=", "==", "!="};
const char* const kCasts[] = {"f32", "f64", "i32", "i64"};

bool in(const char* const* list, size_t n, const std::string& s) {
  for (size_t k = 0; k < n; ++k)
    if (s == list[k]) return true;
  return false;
}
#define PYC_IN(list, s) in(list, sizeof(list) / sizeof(list[0]), s)

VT leaf_type(pyc_dtype d) {
  switch (d) {
    case PYC_F32: case PYC_BF16: case PYC_F16: return VT::F32;
    case PYC_F64: return VT::F64;
    case PYC_I32: return VT::I32;
    case PYC_I64: return VT::I64;
    default: fail(PYC_E_ARG, "expression arguments are F32, F64, BF16, F16, I32 or I64");
  }
}

// Result type of combining a and b: the wider one; a weak literal adopts the other
// side's type, except that a fractional literal with an integer side gives double.
VT promote(const Node& a, const Node& b) {
  if (a.weak && !b.weak) {
    if (a.type == VT::F64 && !vt_float(b.type)) return VT::F64;
    return b.type;
  }
  if (b.weak && !a.weak) {
    if (b.type == VT::F64 && !vt_float(a.type)) return VT::F64;
    return a.type;
  }
  return (int)a.type > (int)b.type ? a.type : b.type;
}

void type_check(Node& n, const std::vector<Arg>& args) {
  if (n.op == "$" || n.op == "%") {
    if (n.slot >= (int)args.size()) fail(PYC_E_PARSE, "expression: argument " +
                                                       std::to_string(n.slot) + " is not declared");
    const Arg& a = args[n.slot];
    if (a.is_array != (n.op == "$"))
      fail(PYC_E_PARSE, "expression: argument " + std::to_string(n.slot) + " is " +
                            (a.is_array ? "an array (use $)" : "a scalar (use %)"));
    n.type = leaf_type(a.dtype);
    return;
  }
  if (n.op == "#") {
    n.type = n.lit_float ? VT::F64 : VT::I32;
    n.weak = true;
    return;
  }
  for (auto& k : n.kids) type_check(*k, args);
  const size_t nk = n.kids.size();
  auto need = [&](size_t k) {
    if (nk != k)
      fail(PYC_E_PARSE, "expression: '" + n.op + "' takes " + std::to_string(k) + " operand(s)");
  };
  if (PYC_IN(kUnary, n.op)) {
    need(1);
    const Node& a = *n.kids[0];
    if (n.op == "neg" || n.op == "abs") {
      n.type = a.type;
      n.weak = a.weak;
    } else {
      n.type = vt_float(a.type) ? a.type : VT::F64;  // integer operands: double
      if (a.weak) n.type = VT::F64, n.weak = true;
    }
  } else if (PYC_IN(kBinary, n.op)) {
    need(2);
    const Node& a = *n.kids[0];
    const Node& b = *n.kids[1];
    VT t = promote(a, b);
    if (n.op == "/" && !vt_float(t)) t = VT::F64;  // true division
    if (n.op == "pow" && !vt_float(t)) t = VT::F64;
    bool cmp = n.op == "<" || n.op == "<=" || n.op == ">" || n.op == ">=" || n.op == "==" ||
               n.op == "!=";
    n.type = cmp ? VT::I32 : t;
    n.weak = !cmp && a.weak && b.weak;
  } else if (n.op == "where") {
    need(3);
    Node& a = *n.kids[1];
    Node& b = *n.kids[2];
    n.type = promote(a, b);
    n.weak = a.weak && b.weak;
  } else if (PYC_IN(kCasts, n.op)) {
    need(1);
    n.type = n.op == "f32" ? VT::F32 : n.op == "f64" ? VT::F64 : n.op == "i32" ? VT::I32 : VT::I64;
  } else {
    fail(PYC_E_PARSE, "expression: unknown operator '" + n.op + "'");
  }
}

std::string literal_as(const Node& n, VT t) {
  double v = std::strtod(n.literal.c_str(), nullptr);
  char buf[64];
  switch (t) {
    case VT::F32: {
      std::snprintf(buf, sizeof buf, "%.9g", (double)(float)v);
      std::string r = buf;
      if (r.find_first_of(".eE") == std::string::npos) r += ".0";
      return r + "f";
    }
    case VT::F64:
      std::snprintf(buf, sizeof buf, "%.17g", v);
      break;
    case VT::I32:
      if (n.lit_float) fail(PYC_E_PARSE, "expression: fractional literal in integer context");
      std::snprintf(buf, sizeof buf, "%lld", (long long)v);
      return std::string("((int)") + buf + ")";
    default:
      if (n.lit_float) fail(PYC_E_PARSE, "expression: fractional literal in integer context");
      std::snprintf(buf, sizeof buf, "%lldLL", (long long)v);
      break;
  }
  std::string r = buf;
  if (t == VT::F64 && r.find_first_of(".eEn") == std::string::npos) r += ".0";
  return r;
}

// C source of n converted to type t.
std::string emit(const Node& n, const std::vector<Arg>& args, VT t);

std::string emit_own(const Node& n, const std::vector<Arg>& args) {
  const std::string T = vt_name(n.type);
  const bool f32 = n.type == VT::F32;
  if (n.op == "$") {
    std::string r = "a" + std::to_string(n.slot) + "[i]";
    pyc_dtype d = args[n.slot].dtype;
    if (d == PYC_BF16 || d == PYC_F16) r = "((float)" + r + ")";
    return r;
  }
  if (n.op == "%") return "a" + std::to_string(n.slot);
  if (n.op == "#") return literal_as(n, n.type);
  if (PYC_IN(kCasts, n.op)) return "((" + T + ")" + emit(*n.kids[0], args, n.kids[0]->type) + ")";
  if (PYC_IN(kUnary, n.op)) {
    std::string a = emit(*n.kids[0], args, n.type);
    if (n.op == "neg") return "(-" + a + ")";
    if (n.op == "abs") {
      if (vt_float(n.type)) return std::string(f32 ? "fabsf(" : "fabs(") + a + ")";
      return "(" + a + " < 0 ? -" + a + " : " + a + ")";
    }
    std::string fn = n.op;
    if (f32) fn += "f";
    return fn + "(" + a + ")";
  }
  if (n.op == "where") {
    std::string c = emit(*n.kids[0], args, n.kids[0]->type);
    return "(" + c + " != 0 ? " + emit(*n.kids[1], args, n.type) + " : " +
           emit(*n.kids[2], args, n.type) + ")";
  }
  // binary: operands converted to the promoted operand type
  const Node& a = *n.kids[0];
  const Node& b = *n.kids[1];
  VT ot = promote(a, b);
  if ((n.op == "/" || n.op == "pow") && !vt_float(ot)) ot = VT::F64;
  std::string x = emit(a, args, ot), y = emit(b, args, ot);
  if (n.op == "min" || n.op == "max") {
    if (vt_float(ot))
      return std::string(n.op == "min" ? "fmin" : "fmax") + (ot == VT::F32 ? "f(" : "(") + x +
             ", " + y + ")";
    return "(" + x + (n.op == "min" ? " < " : " > ") + y + " ? " + x + " : " + y + ")";
  }
  if (n.op == "pow") return std::string(ot == VT::F32 ? "powf(" : "pow(") + x + ", " + y + ")";
  if (n.op == "+" || n.op == "-" || n.op == "*" || n.op == "/") {
    if (!vt_float(ot) && n.op != "/")  // integers wrap (two's complement), as in the reduction
      return "((" + std::string(vt_name(ot)) + ")((" +
             std::string(ot == VT::I32 ? "unsigned" : "unsigned long long") + ")" + x + " " +
             n.op + " (" + std::string(ot == VT::I32 ? "unsigned" : "unsigned long long") + ")" +
             y + "))";
    return "(" + x + " " + n.op + " " + y + ")";
  }
  return "(" + x + " " + n.op + " " + y + " ? 1 : 0)";  // comparison
}

std::string emit(const Node& n, const std::vector<Arg>& args, VT t) {
  if (n.op == "#") return literal_as(n, t);
  std::string s = emit_own(n, args);
  if (n.type == t) return s;
  return "((" + std::string(vt_name(t)) + ")" + s + ")";
}

const char* spec_name(pyc_dtype d) {
  switch (d) {
    case PYC_F32: return "float";
    case PYC_F64: return "double";
    case PYC_BF16: return "__nv_bfloat16";
    case PYC_F16: return "__half";
    case PYC_I32: return "int";
    case PYC_I64: return "long long";
    default: fail(PYC_E_ARG, "unsupported dtype in an expression");
  }
}

VT vt_of_dtype(pyc_dtype d) { return leaf_type(d); }

struct Compiled {
  std::string argspec;  // a0 .. a{n-1}[, out]
  std::string expr;     // C expression of the value, in the type `type`
  VT type;
};

Compiled compile(const char* text, int nargs, const pyc_dtype* dtypes, const int* is_array,
                 bool with_out, pyc_dtype out_dtype) {
  if (!text) fail(PYC_E_ARG, "expr is NULL");
  if (nargs < 0 || (nargs > 0 && (!dtypes || !is_array)))
    fail(PYC_E_ARG, "argument descriptions are missing");
  std::vector<Arg> args;
  for (int k = 0; k < nargs; ++k) args.push_back(Arg{dtypes[k], is_array[k] != 0});
  std::string s = text;
  Parser ps(s);
  std::unique_ptr<Node> root = ps.parse();
  ps.skip();
  if (ps.p != s.size()) ps.error("trailing text");
  type_check(*root, args);
  Compiled c;
  for (int k = 0; k < nargs; ++k) {
    if (k) c.argspec += ", ";
    c.argspec += std::string(spec_name(args[k].dtype)) + (args[k].is_array ? " *a" : " a") +
                 std::to_string(k);
  }
  c.type = with_out ? vt_of_dtype(out_dtype) : root->type;
  if (root->weak && !with_out) c.type = root->type;
  if (with_out) c.argspec += std::string(nargs ? ", " : "") + spec_name(out_dtype) + " *out";
  c.expr = emit(*root, args, c.type);
  return c;
}

}  // namespace

}  // namespace pyc

using namespace pyc;

PYC_API pyc_status pyc_expr_map_create(const char* expr, int nargs, const pyc_dtype* arg_dtypes,
                                       const int* arg_is_array, pyc_dtype out_dtype,
                                       const pyc_opts* opts, pyc_map_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    Compiled c = compile(expr, nargs, arg_dtypes, arg_is_array, true, out_dtype);
    std::string stmt = "out[i] = " + c.expr;
    pyc_status st = pyc_map_create(c.argspec.c_str(), stmt.c_str(), "expr", opts, out);
    if (st != PYC_OK) throw Error(st, pyc_last_error());
  });
}

PYC_API pyc_status pyc_expr_reduce_create(const char* expr, int nargs,
                                          const pyc_dtype* arg_dtypes, const int* arg_is_array,
                                          pyc_dtype out_dtype, const char* reduce,
                                          const pyc_opts* opts, pyc_reduce_t* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!reduce) fail(PYC_E_ARG, "reduce is NULL");
    std::string r = reduce;
    if (out_dtype != PYC_F32 && out_dtype != PYC_F64 && out_dtype != PYC_I32 &&
        out_dtype != PYC_I64)
      fail(PYC_E_ARG, "an expression reduction's result is F32, F64, I32 or I64");
    Compiled c = compile(expr, nargs, arg_dtypes, arg_is_array, false, out_dtype);
    const bool flt = out_dtype == PYC_F32 || out_dtype == PYC_F64;
    const std::string T = type_info(out_dtype).device_name;
    std::string neutral, op;
    if (r == "sum") {
      neutral = "0";
      op = "a+b";
    } else if (r == "max") {
      neutral = flt ? "-INFINITY" : (out_dtype == PYC_I32 ? "(-2147483647-1)" : "(-9223372036854775807LL-1)");
      op = "a > b ? a : b";
    } else if (r == "min") {
      neutral = flt ? "INFINITY" : (out_dtype == PYC_I32 ? "2147483647" : "9223372036854775807LL");
      op = "a < b ? a : b";
    } else {
      fail(PYC_E_ARG, "reduce is \"sum\", \"max\" or \"min\"");
    }
    std::string mexpr = "(" + T + ")" + c.expr;
    pyc_status st = pyc_reduce_create(out_dtype, neutral.c_str(), op.c_str(), mexpr.c_str(),
                                      c.argspec.c_str(), opts, out);
    if (st != PYC_OK) throw Error(st, pyc_last_error());
  });
}

PYC_API pyc_status pyc_expr_type(const char* expr, int nargs, const pyc_dtype* arg_dtypes,
                                 const int* arg_is_array, pyc_dtype* out) {
  return guarded([&] {
    if (!out) fail(PYC_E_ARG, "out is NULL");
    Compiled c = compile(expr, nargs, arg_dtypes, arg_is_array, false, PYC_F32);
    *out = c.type == VT::I32 ? PYC_I32 : c.type == VT::I64 ? PYC_I64
         : c.type == VT::F32 ? PYC_F32 : PYC_F64;
  });
}
