// GENERATED by gen_sbox_circuit.py -- do not edit.
// The AES S-box (FIPS-197 section 5.1.1) as a straight-line circuit on
// 32-bit words: bit k of x_i is bit i of the k-th of 32 independent inputs.
// Composite field GF(((2^2)^2)^2); bases (poly: a1 t + a0, t^2 = t + c; normal:
// a1 T + a0 T^q, T^2 = T + c) and constants c of GF(4), GF(16), GF(256):
// tower = normal 1, normal 1, normal 2; beta = 0x65; tie-break seed = 82;
// 36 AND + 100 XOR gates, plus NOTs for the affine constant 0x63
// (the compiler merges them into three-input LOP3 operations).
#pragma once
#include <cstdint>

namespace kgpu {

__device__ __forceinline__ void sbox_circuit(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                             uint32_t& x4, uint32_t& x5, uint32_t& x6, uint32_t& x7) {
    const uint32_t n53 = x2 ^ x4;
    const uint32_t n0 = x1 ^ x3;
    const uint32_t n3 = x2 ^ n0;
    const uint32_t n15 = x6 ^ n3;
    const uint32_t n2 = x4 ^ x7;
    const uint32_t g1 = n15 & n2;
    const uint32_t n8 = g1 ^ n3;
    const uint32_t n1 = x5 ^ x6;
    const uint32_t n9 = n0 ^ n2;
    const uint32_t n29 = x2 ^ n2;
    const uint32_t n39 = x1 ^ n29;
    const uint32_t g3 = n9 & n39;
    const uint32_t n22 = x4 ^ g3;
    const uint32_t n23 = n1 ^ n22;
    const uint32_t n58 = n1 ^ n9;
    const uint32_t n25 = x2 ^ x7;
    const uint32_t g2 = n58 & n25;
    const uint32_t n4 = x0 ^ n1;
    const uint32_t n51 = x4 ^ n4;
    const uint32_t g4 = x0 & n51;
    const uint32_t n24 = g2 ^ g4;
    const uint32_t n43 = n23 ^ n24;
    const uint32_t n49 = n8 ^ n43;
    const uint32_t n74 = x5 ^ n3;
    const uint32_t n46 = x1 ^ x7;
    const uint32_t g6 = n74 & n46;
    const uint32_t n64 = x5 ^ n29;
    const uint32_t g0 = n64 & n53;
    const uint32_t n48 = x0 ^ n9;
    const uint32_t n17 = x1 ^ n4;
    const uint32_t n65 = n17 ^ n25;
    const uint32_t g5 = n48 & n65;
    const uint32_t n11 = g0 ^ g5;
    const uint32_t n12 = g3 ^ n2;
    const uint32_t n14 = x6 ^ n12;
    const uint32_t n72 = n11 ^ n14;
    const uint32_t n79 = n8 ^ n72;
    const uint32_t n5 = x5 ^ x7;
    const uint32_t n26 = g6 ^ n5;
    const uint32_t g8 = n4 & n17;
    const uint32_t n40 = g1 ^ g8;
    const uint32_t n42 = x2 ^ n40;
    const uint32_t n47 = g0 ^ n42;
    const uint32_t n63 = n26 ^ n47;
    const uint32_t n67 = x3 ^ n63;
    const uint32_t g11 = n79 & n67;
    const uint32_t n20 = g6 ^ g11;
    const uint32_t n45 = n5 ^ n11;
    const uint32_t n55 = n24 ^ n45;
    const uint32_t n7 = x1 ^ g8;
    const uint32_t n57 = x0 ^ n15;
    const uint32_t n50 = x7 ^ n4;
    const uint32_t g7 = n57 & n50;
    const uint32_t n34 = g2 ^ g7;
    const uint32_t n71 = n7 ^ n34;
    const uint32_t n76 = g0 ^ n71;
    const uint32_t g9 = n55 & n76;
    const uint32_t n18 = g9 ^ n7;
    const uint32_t n33 = g5 ^ n18;
    const uint32_t n69 = n23 ^ n33;
    const uint32_t n70 = n20 ^ n69;
    const uint32_t g16 = n49 & n70;
    const uint32_t n73 = n26 ^ n34;
    const uint32_t n78 = n8 ^ n73;
    const uint32_t g10 = n49 & n78;
    const uint32_t n19 = g4 ^ g10;
    const uint32_t n31 = g7 ^ n19;
    const uint32_t n75 = n5 ^ n33;
    const uint32_t n77 = n31 ^ n75;
    const uint32_t g17 = n79 & n77;
    const uint32_t n13 = g16 ^ g17;
    const uint32_t g13 = n78 & n70;
    const uint32_t g14 = n67 & n77;
    const uint32_t n21 = g13 ^ g14;
    const uint32_t n52 = n13 ^ n21;
    const uint32_t g18 = n53 & n52;
    const uint32_t n54 = n20 ^ n31;
    const uint32_t n60 = n14 ^ n54;
    const uint32_t g12 = n76 & n60;
    const uint32_t n28 = g12 ^ g13;
    const uint32_t g15 = n55 & n60;
    const uint32_t n32 = g15 ^ g16;
    const uint32_t n56 = n28 ^ n32;
    const uint32_t g19 = n2 & n56;
    const uint32_t n6 = g18 ^ g19;
    const uint32_t n16 = g15 ^ g17;
    const uint32_t g26 = n17 & n16;
    const uint32_t g34 = n57 & n32;
    const uint32_t n44 = g26 ^ g34;
    const uint32_t n59 = n6 ^ n44;
    const uint32_t g33 = n74 & n13;
    const uint32_t g30 = n9 & n21;
    const uint32_t g24 = n46 & n13;
    const uint32_t g31 = x0 & n28;
    const uint32_t n36 = g24 ^ g31;
    const uint32_t n38 = g30 ^ n36;
    const uint32_t n80 = g33 ^ n38;
    const uint32_t n97 = n59 ^ n80;
    const uint32_t n27 = g12 ^ g14;
    const uint32_t n66 = n16 ^ n27;
    const uint32_t g29 = n58 & n66;
    const uint32_t n90 = g24 ^ g29;
    const uint32_t g27 = n64 & n52;
    const uint32_t g35 = n4 & n16;
    const uint32_t n89 = g35 ^ n59;
    const uint32_t n94 = g27 ^ n89;
    const uint32_t n96 = n90 ^ n94;
    const uint32_t g22 = n51 & n28;
    const uint32_t g25 = n50 & n32;
    const uint32_t n41 = g25 ^ g29;
    const uint32_t n61 = n38 ^ n41;
    const uint32_t g23 = n65 & n27;
    const uint32_t n10 = g23 ^ n6;
    const uint32_t n37 = g33 ^ g35;
    const uint32_t n85 = n10 ^ n37;
    const uint32_t n86 = n61 ^ n85;
    const uint32_t n91 = g22 ^ n86;
    const uint32_t n99 = g27 ^ n91;
    const uint32_t g32 = n48 & n27;
    const uint32_t g21 = n39 & n21;
    const uint32_t n30 = g21 ^ n10;
    const uint32_t n35 = g32 ^ n30;
    const uint32_t n81 = g31 ^ n35;
    const uint32_t n82 = g34 ^ g35;
    const uint32_t n87 = n81 ^ n82;
    const uint32_t n68 = g30 ^ n35;
    const uint32_t n88 = n37 ^ n68;
    const uint32_t g28 = n15 & n56;
    const uint32_t g20 = n25 & n66;
    const uint32_t n83 = g19 ^ n61;
    const uint32_t n93 = g20 ^ n83;
    const uint32_t n98 = g28 ^ n93;
    const uint32_t n62 = g27 ^ g28;
    const uint32_t n95 = n62 ^ n68;
    const uint32_t n84 = n30 ^ n37;
    const uint32_t n92 = n62 ^ n84;
    x0 = ~n97;
    x1 = ~n96;
    x2 = n99;
    x3 = n87;
    x4 = n88;
    x5 = ~n98;
    x6 = ~n95;
    x7 = n92;
}

}  // namespace kgpu
