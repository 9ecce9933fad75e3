// Generated by gen_dp5_nystrom.py from the Dormand-Prince 5(4) tableau. Do not edit.
#pragma once

// stage nodes c_s
#define DP_C1 0.0
#define DP_C2 0.2
#define DP_C3 0.3
#define DP_C4 0.8
#define DP_C5 0.8888888888888888
#define DP_C6 1.0
#define DP_C7 1.0
// (A A)_{sm}: h^2 weights of accelerations in stage positions (stage s = 1..7, m = 1..s-2)
#define DP_AA31 0.045
#define DP_AA41 -0.48
#define DP_AA42 0.8
#define DP_AA51 -1.8667885992988873
#define DP_AA52 3.2958390489254685
#define DP_AA53 -1.0339887212315195
#define DP_AA61 -2.018939393939394
#define DP_AA62 4.136363636363637
#define DP_AA63 -1.696969696969697
#define DP_AA64 0.07954545454545454
#define DP_AA71 0.09114583333333333
#define DP_AA73 0.31446540880503143
#define DP_AA74 0.13020833333333334
#define DP_AA75 -0.03581957547169811
// b: fifth-order velocity weights (b2 = b7 = 0)
#define DP_B1 0.09114583333333333
#define DP_B3 0.44923629829290207
#define DP_B4 0.6510416666666666
#define DP_B5 -0.322376179245283
#define DP_B6 0.13095238095238096
// b - bhat: embedded error weights on accelerations (velocity error)
#define DP_E1 0.0012326388888888888
#define DP_E3 -0.0042527702905061394
#define DP_E4 0.03697916666666667
#define DP_E5 -0.05086379716981132
#define DP_E6 0.0419047619047619
#define DP_E7 -0.025
// (b - bhat) A: embedded error weights on accelerations (position error, times h^2)
#define DP_EA1 0.002651909722222222
#define DP_EA3 -0.006157532195268044
#define DP_EA4 0.010182291666666666
#define DP_EA5 -0.003402859669811321
#define DP_EA6 -0.003273809523809524
// continuous extension: velocity weights b_j(s) = sum_p BI_jp s^(p+1)
#define DP_BI11 1.0
#define DP_BI12 -2.859375
#define DP_BI13 3.0833333333333335
#define DP_BI14 -1.1328125
#define DP_BI32 4.0431266846361185
#define DP_BI33 -6.289308176100629
#define DP_BI34 2.6954177897574123
#define DP_BI42 -3.90625
#define DP_BI43 10.416666666666666
#define DP_BI44 -5.859375
#define DP_BI52 2.7939268867924527
#define DP_BI53 -6.877358490566038
#define DP_BI54 3.761055424528302
#define DP_BI62 -1.5714285714285714
#define DP_BI63 3.6666666666666665
#define DP_BI64 -1.9642857142857142
#define DP_BI72 1.5
#define DP_BI73 -4.0
#define DP_BI74 2.5
// continuous extension: position weights P_m(s) = sum_p PX_mp s^(p+1), times h^2
#define DP_PX12 0.3971354166666667
#define DP_PX13 -0.5208333333333334
#define DP_PX14 0.21484375
#define DP_PX32 0.23360287511230907
#define DP_PX33 0.3414195867026056
#define DP_PX34 -0.2605570530098832
#define DP_PX42 -0.2734375
#define DP_PX43 0.4166666666666667
#define DP_PX44 -0.013020833333333334
#define DP_PX52 -0.05372936320754717
#define DP_PX53 0.2865566037735849
#define DP_PX54 -0.2686468160377358
#define DP_PX62 0.19642857142857142
#define DP_PX63 -0.5238095238095238
#define DP_PX64 0.3273809523809524
