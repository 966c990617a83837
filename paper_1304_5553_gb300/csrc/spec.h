// Argument-spec parsing and statement analysis.
//
// An argument spec is a C parameter list (Sec. 3.2.4, Listing 3a):
// "float a, float *x, float b, float *y, float *z".  Pointers are arrays
// indexed by the formal index i; everything else is a scalar passed by value.
// The statement (map) or expression (map-reduce) is C code in i.
//
// The analysis decides, per array, whether the code only ever touches it as
// name[i].  Such arrays are "lifted": the generated kernel moves them through
// registers with wide vector loads and stores, and the code's name[i] is
// rewritten to the register copy.  Arrays used any other way stay raw
// pointers.  A lifted array is loaded if the code may read it or may leave an
// element unwritten, and stored if the code may write it.
#pragma once

#include <string>
#include <vector>

#include "common.h"

namespace pyc {

struct Param {
  std::string name;
  pyc_dtype dtype = PYC_F32;
  bool is_ptr = false;
  bool is_const = false;
  int scalar_offset = -1;  // offset in the packed scalar block
  int ptr_slot = -1;       // index in ptrs[]
  int args_offset = 0;     // offset in the device-side argument struct
  // analysis (arrays only)
  bool used = false;
  bool read = false;
  bool written = false;
  bool lifted = false;
  bool raw = false;            // used other than as name[i] somewhere
  bool fully_written = false;  // some top-level statement assigns name[i] unconditionally
};

struct ArgSpec {
  std::vector<Param> params;
  int scalar_bytes = 0;  // size of the packed scalar block
  int num_ptrs = 0;
  int args_bytes = 0;    // size of the device-side argument struct
  int args_align = 1;
  std::string canonical;  // normalised text, part of the cache key
};

// Parses a C parameter list; throws Error(PYC_E_PARSE).
ArgSpec parse_argspec(const std::string& text);

struct Token {
  enum Kind { Ident, Number, String, Punct } kind;
  std::string text;
};

// Tokenises C code (comments dropped); throws Error(PYC_E_PARSE) on
// preprocessor lines, unterminated literals/comments or stray characters.
std::vector<Token> tokenize(const std::string& code);

// Analyses `code` against the arrays of `spec` (updating their flags, which
// accumulate over several calls) and returns the code with every lifted
// access name[i] replaced by pyc_r_<name>[pyc_k].  `expression` = true for
// a map-reduce map expression (writes make an array raw).  Throws
// Error(PYC_E_PARSE) on unbalanced brackets or forbidden constructs.
std::string analyze_and_rewrite(ArgSpec& spec, const std::string& code, bool expression);

// The two halves of analyze_and_rewrite, for specs with several pieces of code
// (analyse every piece first, then rewrite each with the final flags).
void analyze_code(ArgSpec& spec, const std::string& code, bool expression);
std::string rewrite_lifted(ArgSpec& spec, const std::string& code);

// Checks an expression that may only use the given formal names (a, b for
// reduce expressions); returns it re-joined from tokens.
std::string check_expression(const std::string& code, const char* what);

// Join tokens back into source text.
std::string join_tokens(const std::vector<Token>& t);

}  // namespace pyc
