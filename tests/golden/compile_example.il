; Sec. 4, Example 3 (compiling contracts to payoffs).
; CL:  translate(t0, both(scale(100.0, transfer(you, me)),
;        translate(t1, if(obs(AAPL,0) > 100.0,
;                         scale(obs(AAPL,0) - 100.0, transfer(you, me)), zero))))
; Expected tau_c output, written exactly as the compiler builds it: translate
; shifts accumulate into t0 through the smart constructor tplus (a numeral 0
; start time and the obs offset 0 stay as tplus operands because t0, t1 are
; template variables), and CL's if is ifWithin with window 0, i.e. loopif(.., 0).
; Names: $0 = t0, $1 = t1, you = 0, me = 1, AAPL = label 0.
(add (mult 100.0 (payoff (tplus 0 $0) 0 1))
     (loopif (lt 100.0 (model 0 (tplus (tplus (tplus 0 $0) $1) 0)))
             (mult (sub (model 0 (tplus (tplus (tplus 0 $0) $1) 0)) 100.0)
                   (payoff (tplus (tplus 0 $0) $1) 0 1))
             0.0
             0))
