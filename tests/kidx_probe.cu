// Host-side probe of the operand K order shared by the block formation (k_s2_form_u, which
// writes U_k's digit planes) and the tensor-core update kernel (which writes the lines' digit
// planes): prints tc_kidx(p) for the 32 window positions.  Built and run by
// tests/test_emu_layout_host.py; no GPU is needed.
#include <cstdio>

#include "../paper_2301_07964_gb300/csrc/emu_arith.cuh"

int main()
{
    for (int p = 0; p < 32; ++p) printf("%d %d\n", p, hts::emu::tc_kidx(p));
    return 0;
}
